// Internal declarations shared by the solver kernels and the C ABI layer.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "hjpdhg.h"

namespace hj {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxD = 128;   // largest state dimension of the families with d x d data
constexpr int kMaxDEik = 4096;   // largest state dimension of the eikonal family
constexpr int kMaxN = 256;   // largest number of time steps

// Everything a solve kernel needs, passed by value.  Scalars that enter the
// iteration are given in double; kernels round them to the iterate type once.
template <typename T>
struct SolveArgs {
  int64_t B;
  int32_t N, d;
  double sigma, tau, theta, tol;
  // tol as an unevaluated sum of two floats (tol_hi = fl32(tol), tol_lo =
  // fl32(tol - tol_hi): within 2^-48 tol), for the FP32 kernels' stopping test
  float tol_hi, tol_lo;
  // The same step sizes rounded once to the iterate type on the host, so the
  // iteration loop holds no double-derived value the compiler could recompute
  // there (FP64 instructions are ~64x the cost of FP32 ones on this GPU).
  T sigma_t, tau_t, theta_t;
  int32_t max_iter, check_every, inner_steps;
  int32_t formulation;   // HJ_FORM_LAX or HJ_FORM_HOPF
  // HJ_SCHEME_*: H on interval j weighted wR at x_j and wL at x_{j-1}
  // (backward Euler 1, 0; forward Euler 0, 1; trapezoid 1/2, 1/2)
  int32_t scheme;
  T mix_wr_t, mix_wl_t;
  double mix_wr, mix_wl;
  // value test (value_tol > 0): stop when fval moved less than value_tol
  // between two tests
  int32_t value_stop;
  double value_tol;
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
  double eik_c0, eik_c1, eik_c2;       // eikonal speed c(x) = c0 + c1 exp(-c2 |x - x_b|^2)
  // the same in the iterate type, rounded once on the host (fill_family_consts):
  // 1/m, a_h, g_z, eps and c0, c1, c2.  A kernel that rematerialises one of them
  // under register pressure then loads it instead of converting a double (an
  // FP64-pipe instruction at 1/64 rate)
  T qc_t[4], eik_t[3];
  const double* xb64;                  // [d] eikonal bump centre x_b
  const T* xb;                         // [d] the same in T
  // eikonal bump moving with velocity v_b: c(x - s v_b) at node time s = j delta
  int32_t eik_moving;
  const double* vb64;                  // [d] v_b (null when static)
  const T* vb;
  // +1, or -1 for the negative eikonal equation: the kernels solve the positive
  // one with the initial data -g (x_0 prox and value with -W^2) and return
  // V and p multiplied by cost_sign
  double cost_sign;
  int32_t game_d1;                     // difference-of-norms game: coordinates of the
                                       // minimising player (d for every other family)
  // budget of the launch (0: none): nanoseconds since its first draw, and
  // iterations of the points finished; when either runs out the remaining
  // points are drained with status HJ_POINT_TIMEOUT
  int64_t budget_ns, iter_budget;
  unsigned long long* counter;        // work counter block, kCounterWords (zeroed before launch)
  // Ragged batches: the launch processes items i = 0..B-1, point id idx[i]
  // (idx null: id = i).  Per-point N (Nv null: N), xq offset in doubles
  // (xq_off null: id*d) and trajectory offset in elements (traj_off null:
  // id*(N+1)*d).  V, iters, status and t are indexed by the point id.
  const int32_t* idx;
  const int32_t* Nv;
  const int64_t* xq_off;
  const int64_t* traj_off;
};

template <typename T>
inline void fill_family_consts(SolveArgs<T>& a) {
  a.qc_t[0] = a.qc_m != 0.0 ? T(1.0 / a.qc_m) : T(0);
  a.qc_t[1] = T(a.qc_ah);
  a.qc_t[2] = T(a.qc_gz);
  a.qc_t[3] = T(a.qc_eps);
  a.eik_t[0] = T(a.eik_c0);
  a.eik_t[1] = T(a.eik_c1);
  a.eik_t[2] = T(a.eik_c2);
}

template <typename T>
struct PointRef {
  int64_t id;
  int N;
  const double* xq;
  size_t traj;      // element offset of the point's [N+1][d] block
};

template <typename T>
__device__ __forceinline__ PointRef<T> point_ref(const SolveArgs<T>& a, int64_t item) {
  PointRef<T> r;
  r.id = a.idx ? (int64_t)a.idx[item] : item;
  r.N = a.Nv ? a.Nv[r.id] : a.N;
  r.xq = a.xq + (a.xq_off ? a.xq_off[r.id] : r.id * (int64_t)a.d);
  r.traj = a.traj_off ? (size_t)a.traj_off[r.id] : (size_t)r.id * (size_t)(r.N + 1) * a.d;
  return r;
}

// The work counter block of a persistent launch, zeroed before the launch:
// [0] the next item to draw, [1] the launch's start time on the global timer
// (set by the first draw when a time budget is on), [2] the iterations of the
// points finished so far (counted when an iteration budget is on).
constexpr int kCounterWords = 3;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// A point drained after the budget ran out: not iterated, V = NaN (one thread).
template <typename T>
__device__ __forceinline__ void mark_timed_out(const SolveArgs<T>& a, int64_t item) {
  const int64_t id = a.idx ? (int64_t)a.idx[item] : item;
  a.status[id] = HJ_POINT_TIMEOUT;
  a.iters[id] = 0;
  a.V[id] = __longlong_as_double(0x7ff8000000000000ll);
}

// Draw the next item to solve (one thread of the group); an item >= B ends the
// launch.  Once the launch's budget has run out, the drawing thread marks each
// item it draws HJ_POINT_TIMEOUT and draws again, so the batch drains without
// the solver loop seeing those items (each draw advances the counter: at most
// B draws).
template <typename T>
__device__ __forceinline__ unsigned long long draw_item(const SolveArgs<T>& a) {
  for (;;) {
    const unsigned long long it = atomicAdd(a.counter, 1ull);
    if (it >= (unsigned long long)a.B || (a.budget_ns <= 0 && a.iter_budget <= 0)) return it;
    bool out = false;
    if (a.budget_ns > 0) {
      const unsigned long long now = global_ns();
      unsigned long long t0 = atomicCAS(a.counter + 1, 0ull, now);
      if (t0 == 0ull) t0 = now;
      out = (long long)(now - t0) > (long long)a.budget_ns;
    }
    if (a.iter_budget > 0)
      out = out || *reinterpret_cast<volatile unsigned long long*>(a.counter + 2) >=
                       (unsigned long long)a.iter_budget;
    if (!out) return it;
    mark_timed_out(a, (int64_t)it);
  }
}

// A finished point's iterations, for the iteration budget (one thread).
template <typename T>
__device__ __forceinline__ void count_iterations(const SolveArgs<T>& a, int k) {
  if (a.iter_budget > 0) atomicAdd(a.counter + 2, (unsigned long long)k);
}

// Launch shape of the register-resident kernel: G warps per point, NPL time
// nodes per lane; a point needs N <= 32 * G * NPL.  half = 1 (with G = 1,
// NPL = 1): half a warp per point, two points per warp, N <= 16.
struct WarpConfig {
  int G, NPL;
  int half = 0;
};
inline int warp_config_lanes(const WarpConfig& c) { return c.half ? 16 : 32 * c.G; }

// splitmix64 (Vigna 2015) evaluated at a counter: z = seed + (c + 1) * golden,
// followed by the generator's xor-shift-multiply finaliser.  Used for the
// random initial guess of Section 6; the counter layout is
// point * 2^32 + stream * 2^31 + j * 2^12 + coord.
__device__ __forceinline__ uint64_t splitmix_at(uint64_t seed, uint64_t point, uint64_t stream,
                                                uint64_t j, uint64_t coord) {
  const uint64_t ctr = (point << 32) + (stream << 31) + (j << 12) + coord;
  uint64_t z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double uniform_pm1(uint64_t seed, uint64_t point, uint64_t stream,
                                              uint64_t j, uint64_t coord) {
  const uint64_t z = splitmix_at(seed, point, stream, j, coord);
  const double u = (double)(z >> 11) * 0x1.0p-53;
  return 2.0 * u - 1.0;
}

// The initial guess of Section 6 in the iterate type: x = x_q + r u and p = r u.
// FP64 evaluates both exactly as written (one rounding each).  FP32 takes the
// generator's top 24 bits as u (exact in FP32, within 2^-23 of the 53-bit u)
// and forms (float)x_q + (float)r * u, so no FP64 instruction runs per value.
template <typename T>
struct InitGuess {
  double r;
  __device__ explicit InitGuess(double radius) : r(radius) {}
  __device__ __forceinline__ T x(double xq, uint64_t seed, uint64_t pt, uint64_t j,
                                 uint64_t k) const {
    return T(xq + r * uniform_pm1(seed, pt, 0, j, k));
  }
  __device__ __forceinline__ T p(uint64_t seed, uint64_t pt, uint64_t j, uint64_t k) const {
    return T(r * uniform_pm1(seed, pt, 1, j, k));
  }
};
template <>
struct InitGuess<float> {
  float r;
  __device__ explicit InitGuess(double radius) : r((float)radius) {}
  __device__ __forceinline__ static float u(uint64_t z) {
    return (float)(uint32_t)(z >> 40) * 0x1.0p-23f - 1.0f;
  }
  __device__ __forceinline__ float x(float xq, uint64_t seed, uint64_t pt, uint64_t j,
                                     uint64_t k) const {
    return __fmaf_rn(r, u(splitmix_at(seed, pt, 0, j, k)), xq);
  }
  __device__ __forceinline__ float p(uint64_t seed, uint64_t pt, uint64_t j, uint64_t k) const {
    return r * u(splitmix_at(seed, pt, 1, j, k));
  }
};

// max that keeps a NaN (fmax drops it): a non-finite residual must not read as small
__device__ __forceinline__ double max_nan(double a, double b) { return (a > b || a != a) ? a : b; }

template <typename U>
__device__ __forceinline__ U warp_sum(U v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// The stopping test's accumulation over a point's warps with FP32 iterates: the
// warps' FP32 sums added as a double-float (an unevaluated sum hi + lo of two
// floats) by Knuth's error-free TwoSum, so the accumulated sum of up to 32
// partials carries about 48 significant bits (relative error a small multiple of
// 2^-48; an FP64 accumulation of the same partials has up to n 2^-53), while
// every instruction runs on the FP32 pipe (an FP64
// instruction holds this GPU's FP64 pipe for about 64 cycles per warp, active
// lanes or not: the FP64 form measured 4 % of the 12-D quadcopter solve).
struct SumF2 {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float b) {
    const float s = hi + b;                 // TwoSum(hi, b) = s + e exactly
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (b - bb);
    const float l = lo + e;
    hi = s + l;                             // renormalise: |s| >= |l| (FastTwoSum)
    lo = l - (hi - s);
  }
  __device__ __forceinline__ void add(const SumF2& o) {   // the same with a double-float
    const float s = hi + o.hi;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (o.hi - bb);
    const float l = (lo + o.lo) + e;
    hi = s + l;
    lo = l - (hi - s);
  }
  // hi + lo < th + tl, up to the rounding of the final difference (2^-48 relative)
  __device__ __forceinline__ bool less(float th, float tl) const {
    return (hi - th) + (lo - tl) < 0.f;
  }
  __device__ __forceinline__ bool finite() const { return isfinite(hi) && isfinite(lo); }
};

// Verdict of a stopping test from n <= 32 per-warp sums (red2[2 w], red2[2 w + 1]:
// warp w's sums of the squared x and p increments), computed by every lane of
// the calling warp: 1 converged (both below tol), 2 non-finite, 0 otherwise.
// FP32: lane w takes warp w's sums and the warp adds them as double-floats by a
// butterfly (TwoSum is exact and symmetric, so every lane ends with the same
// total); FP64: the same butterfly in FP64.
template <typename T>
__device__ __forceinline__ int stop_verdict_lanes(const SolveArgs<T>& a, T vx, T vp);

template <typename T>
__device__ __forceinline__ int stop_verdict(const SolveArgs<T>& a, const T* red2, int n, int lane) {
  return stop_verdict_lanes<T>(a, lane < n ? red2[2 * lane] : T(0), lane < n ? red2[2 * lane + 1] : T(0));
}

// The same with each lane holding one warp's pair of sums (zeros past the last).
template <typename T>
__device__ __forceinline__ int stop_verdict_lanes(const SolveArgs<T>& a, T vx, T vp) {
  if constexpr (sizeof(T) == 4) {
    SumF2 x, p;
    x.hi = vx; p.hi = vp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      SumF2 ox, op;
      ox.hi = __shfl_xor_sync(kFull, x.hi, o); ox.lo = __shfl_xor_sync(kFull, x.lo, o);
      op.hi = __shfl_xor_sync(kFull, p.hi, o); op.lo = __shfl_xor_sync(kFull, p.lo, o);
      x.add(ox);
      p.add(op);
    }
    if (!(x.finite() && p.finite())) return 2;
    return (x.less(a.tol_hi, a.tol_lo) && p.less(a.tol_hi, a.tol_lo)) ? 1 : 0;
  } else {
    double x = vx, p = vp;
    x = warp_sum<double>(x);
    p = warp_sum<double>(p);
    if (!(isfinite(x) && isfinite(p))) return 2;
    return (x < a.tol && p < a.tol) ? 1 : 0;
  }
}

// The same for a compile-time number of warps G (every lane adds the G sums in order).
template <int G, typename T>
__device__ __forceinline__ int stop_verdict_g(const SolveArgs<T>& a, const T* red2) {
  if constexpr (sizeof(T) == 4) {
    SumF2 x, p;
#pragma unroll
    for (int w = 0; w < G; ++w) { x.add(red2[2 * w]); p.add(red2[2 * w + 1]); }
    if (!(x.finite() && p.finite())) return 2;
    return (x.less(a.tol_hi, a.tol_lo) && p.less(a.tol_hi, a.tol_lo)) ? 1 : 0;
  } else {
    double x = 0.0, p = 0.0;
#pragma unroll
    for (int w = 0; w < G; ++w) { x += red2[2 * w]; p += red2[2 * w + 1]; }
    if (!(isfinite(x) && isfinite(p))) return 2;
    return (x < a.tol && p < a.tol) ? 1 : 0;
  }
}

// The same verdict for a point held by one warp (or half-warp): its own sums.
template <typename T>
__device__ __forceinline__ int stop_verdict1(const SolveArgs<T>& a, T x, T p) {
  if (!(isfinite(x) && isfinite(p))) return 2;
  if constexpr (sizeof(T) == 4) {
    SumF2 sx, sp;
    sx.hi = x; sp.hi = p;
    return (sx.less(a.tol_hi, a.tol_lo) && sp.less(a.tol_hi, a.tol_lo)) ? 1 : 0;
  } else {
    return (x < a.tol && p < a.tol) ? 1 : 0;
  }
}

template <typename T>
__device__ __forceinline__ bool finite_val(T v) { return isfinite(v); }

// Arguments of the value-gradient kernel (value_grad.cu).
template <typename T>
struct GradArgs {
  int64_t B;
  int32_t N, d, n_dyn;
  const double* t;
  const T* X;            // [B][N+1][d]
  const T* P;            // [B][N+1][d]
  const double* w;       // [B] dL/dV
  const double* W;       // [d]
  const double* W2;      // [d]
  const double* c;       // [d]
  const T* A;            // tanh drift [d][d]
  double qc_m, qc_ah, qc_gz, qc_eps;
  // eikonal: V = cost_sign V_int, speed c(x - s v_b) = c0 + c1 exp(-c2 |x - s v_b - x_b|^2)
  double cost_sign, eik_c0, eik_c1, eik_c2;
  const double* xb64;    // [d]
  const double* vb64;    // [d] or null (static bump)
  double* dW;            // [d]      accumulated (atomicAdd)
  double* dc;            // [d]
  double* ddyn;          // [n_dyn]
  double* dxq;           // [B][d] or null (written)
};

template <typename T>
hj_status launch_value_grad(int family, const GradArgs<T>& g, cudaStream_t s);

// Reverse sweep through the iterations (adjoint.cu).
template <typename T>
struct AdjArgs {
  int64_t B;
  int32_t N, d, K_cap, C;          // iterations bound, checkpoint spacing
  T sig, tau, th;
  double radius;
  uint64_t seed;
  int64_t point_offset;
  const double* xq;                // [B][d]
  const double* t;                 // [B]
  const int32_t* iters;            // [B] K_b
  const double* w;                 // [B] dL/dV_b
  const double* W2;                // [d]
  const double* W;                 // [d]
  const double* c;                 // [d]
  double qc_m, qc_ah, qc_gz, qc_eps;
  T* work;                         // per CTA: (K_cap / C + 1) checkpoints of 3 (N+1) d
  double* dW;                      // [d]
  double* dc;                      // [d]
  double* ddyn;                    // [4] quadcopter (m, a_h, g_z, eps)
  double* dxq;                     // [B][d]; NaN for a point whose K_b is outside 0..K_cap
  unsigned long long* counter;
};

template <typename T>
hj_status launch_adjoint(int family, const AdjArgs<T>& a, int grid, cudaStream_t s);
int adjoint_grid(int64_t B);

// Kernel launchers (one per kernel family), defined in their .cu files.
// Each returns HJ_OK, HJ_ERR_UNSUPPORTED (no instantiation for this shape) or
// HJ_ERR_CUDA.
template <typename T>
hj_status launch_warp_solver(int family, const SolveArgs<T>& a, WarpConfig cfg, cudaStream_t s);
template <typename T>
hj_status launch_warp_quadratic(const SolveArgs<T>& a, WarpConfig cfg, cudaStream_t s);
template <typename T>
hj_status launch_warp_quadcopter(const SolveArgs<T>& a, WarpConfig cfg, cudaStream_t s);
template <typename T>
hj_status launch_warp_tanh(const SolveArgs<T>& a, WarpConfig cfg, cudaStream_t s);
// the same launchers for the Hopf form (Algorithm 2)
template <typename T>
hj_status launch_warp_quadratic_hopf(const SolveArgs<T>& a, WarpConfig cfg, cudaStream_t s);
template <typename T>
hj_status launch_warp_quadcopter_hopf(const SolveArgs<T>& a, WarpConfig cfg, cudaStream_t s);
template <typename T>
hj_status launch_warp_tanh_hopf(const SolveArgs<T>& a, WarpConfig cfg, cudaStream_t s);
template <typename T>
hj_status launch_warp_eikonal(const SolveArgs<T>& a, WarpConfig cfg, cudaStream_t s);
// forward-Euler and trapezoid schemes (SolveArgs::scheme != HJ_SCHEME_BE)
template <typename T>
hj_status launch_warp_quadcopter_mix(const SolveArgs<T>& a, WarpConfig cfg, cudaStream_t s);
template <typename T>
hj_status launch_warp_tanh_mix(const SolveArgs<T>& a, WarpConfig cfg, cudaStream_t s);
template <typename T>
hj_status launch_warp_eikonal_mix(const SolveArgs<T>& a, WarpConfig cfg, cudaStream_t s);
template <typename T>
hj_status launch_warp_game_mix(const SolveArgs<T>& a, WarpConfig cfg, cudaStream_t s);
template <typename T>
hj_status launch_warp_eikonal_moving(const SolveArgs<T>& a, WarpConfig cfg, cudaStream_t s);
template <typename T>
hj_status launch_warp_game(const SolveArgs<T>& a, WarpConfig cfg, cudaStream_t s);
// Default launch shape for (family, d, Nmax); {0, 0} when no warp kernel fits.
WarpConfig default_warp_config(int family, int d, int Nmax, bool fp64);
// Whether the warp kernel has an instantiation for (family, d, cfg, precision).
bool warp_config_available(int family, int d, WarpConfig cfg, bool fp64);
// Shared-memory CTA kernel: tanh drift (drift = true) or H = |p|^2/2 (drift = false).
// Coordinate-parallel eikonal kernel (any d): one CTA per point, state in shared
// memory when eik_cta_smem_bytes(d, N) != 0, else in a stream-ordered workspace.
template <typename T>
hj_status launch_eik_cta_solver(const SolveArgs<T>& a, cudaStream_t s);
template <typename T>
size_t eik_cta_smem_bytes(int d, int N);
// The same with the state in registers (backward Euler, static bump; FP32:
// d <= 2048 with N <= 10, on a cluster of two CTAs above d = 1024, and d <= 512
// with N <= 16; FP64: d <= 512 with N <= 10); HJ_ERR_UNSUPPORTED elsewhere (the
// shared-memory kernel then runs).
template <typename T>
hj_status launch_eik_reg_solver(const SolveArgs<T>& a, cudaStream_t s);

// Register-tiled FP32 tanh-drift kernel; HJ_ERR_UNSUPPORTED where it does not
// apply (the shared-memory kernel then runs).  td_tile_group_warps: warps per
// point for (d, N), 0 when the tiled kernel cannot hold the point.
hj_status launch_td_tile_solver(const SolveArgs<float>& a, cudaStream_t s);
int td_tile_group_warps(int d, int N);

template <typename T>
hj_status launch_td_cta_solver(const SolveArgs<T>& a, bool drift, cudaStream_t s);
// Shared memory that kernel needs for (d, N) (mix: the forward-Euler /
// trapezoid schemes' extra state array); 0 if it does not fit.
template <typename T>
size_t td_cta_smem_bytes(int d, int N, bool drift, bool mix = false);

}  // namespace hj
