// Internal declarations shared by the solver kernels and the C ABI layer.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "hjpdhg.h"

namespace hj {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxD = 128;   // largest state dimension any kernel accepts
constexpr int kMaxN = 256;   // largest number of time steps

// Everything a solve kernel needs, passed by value.  Scalars that enter the
// iteration are given in double; kernels round them to the iterate type once.
template <typename T>
struct SolveArgs {
  int64_t B;
  int32_t N, d;
  double sigma, tau, theta, tol;
  int32_t max_iter, check_every, inner_steps;
  uint64_t seed;
  double radius;
  int64_t point_offset;
  const double* xq;      // [B][d]
  const double* t;       // [B]
  double* V;             // [B]
  int32_t* iters;        // [B]
  int8_t* status;        // [B]
  T* traj_x;             // [B][N+1][d] or null
  T* traj_p;             // [B][N+1][d] or null
  const T* warm_x;       // [B][N+1][d] or null
  const T* warm_p;       // [B][N+1][d] or null
  const double* W2;      // [d] squared cost weights
  const double* c;       // [d] cost centre
  const T* A;            // tanh drift: [d][d] row-major in T
  const T* At;           // tanh drift: transpose of A in T
  const double* A64;     // tanh drift: [d][d] row-major in double (value epilogue)
  double qc_m, qc_ah, qc_gz, qc_eps;   // quadcopter parameters
  unsigned long long* counter;        // work counter (zeroed before launch)
};

// splitmix64 (Vigna 2015) evaluated at a counter: z = seed + (c + 1) * golden,
// followed by the generator's xor-shift-multiply finaliser.  Used for the
// random initial guess of Section 6; the counter layout is
// point * 2^32 + stream * 2^31 + j * 2^12 + coord.
__device__ __forceinline__ double uniform_pm1(uint64_t seed, uint64_t point, uint64_t stream,
                                              uint64_t j, uint64_t coord) {
  const uint64_t ctr = (point << 32) + (stream << 31) + (j << 12) + coord;
  uint64_t z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= (z >> 31);
  const double u = (double)(z >> 11) * 0x1.0p-53;
  return 2.0 * u - 1.0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ bool finite_val(T v) { return isfinite(v); }

// Kernel launchers (one per kernel family), defined in their .cu files.
// Each returns HJ_OK, HJ_ERR_UNSUPPORTED (no instantiation for this shape) or
// HJ_ERR_CUDA.
template <typename T>
hj_status launch_warp_solver(int family, const SolveArgs<T>& a, cudaStream_t s);
template <typename T>
hj_status launch_td_cta_solver(const SolveArgs<T>& a, cudaStream_t s);
// Shared memory the tanh-drift CTA kernel needs for (d, N); 0 if unsupported.
template <typename T>
size_t td_cta_smem_bytes(int d, int N);

}  // namespace hj
