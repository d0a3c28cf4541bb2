// Residual of the discrete characteristic equations, one thread per (point, node),
// for the families and dimensions the register-resident solver serves
// (quadratic d <= 4, quadcopter, tanh drift d in {2, 4}, eikonal d in {2, 10}).
//
// Thread (b, j), j = 1..N, loads x_j, x_{j-1}, p_j, p_{j+1} of point b from the
// trajectories (a node's d values are contiguous, so consecutive threads read
// consecutive blocks) and evaluates the family's node residual (in FP64, except
// the quadcopter's for FP32 iterates, which is evaluated in FP32)
// (families.cuh kkt_node: max_k |x_j - x_{j-1} - delta grad_p H(x_j, p_j)| and
// |p_{j+1} - p_j + delta grad_x H(x_j, p_j)|; the thread of node 1 adds
// |p_1 - grad g(x_0)|).  The lanes of a warp that hold nodes of the same point
// (a contiguous run of lanes) take their maximum by shuffles, and the run's
// first lane folds it into kkt[b] by an atomic max on the bit pattern of the
// non-negative double (NaN, whose pattern exceeds every finite value's and
// infinity's, wins), so kkt[] is zeroed first.
// Costates are taken in the solver's variables (cost_sign: the negative eikonal
// equation is solved as psi = -phi with initial data -g, Section 6.1).
#include <cuda_runtime.h>

#include <type_traits>

#include "families.cuh"
#include "hj_internal.cuh"
#include "problem.cuh"

namespace hj {

namespace {

// whether the family evaluates its node residual in the iterate type (F::kKktInIterType)
template <class F, class = void>
struct kkt_in_iter_type : std::false_type {};
template <class F>
struct kkt_in_iter_type<F, std::void_t<decltype(F::kKktInIterType)>>
    : std::integral_constant<bool, F::kKktInIterType> {};

// the residual of node j of point b (and, for j = 1, of x_0's equation)
template <typename T, class F, int D>
__device__ __forceinline__ double node_residual(const SolveArgs<T>& a, const F& fam,
                                                     const T* __restrict__ X,
                                                     const T* __restrict__ P, int64_t b, int j,
                                                     const T* __restrict__ gsh) {
  const int N = a.N;
  const double sgn = a.cost_sign;
  {
    const T* xb = X + (size_t)b * (N + 1) * D;
    const T* pb = P + (size_t)b * (N + 1) * D;
    T x[D], xl[D], p[D], pr[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      x[k] = xb[(size_t)j * D + k];
      xl[k] = xb[(size_t)(j - 1) * D + k];
      p[k] = T(sgn) * pb[(size_t)j * D + k];
      pr[k] = j < N ? T(sgn) * pb[(size_t)(j + 1) * D + k] : T(0);
    }
    // families that evaluate FP32 iterates in FP32 take delta = t / N in FP32
    const double delta = (sizeof(T) == 4 && kkt_in_iter_type<F>::value)
                             ? (double)((float)a.t[b] / (float)N) : a.t[b] / N;
    double r = fam.kkt_node(x, xl, p, pr, delta, (double)j * delta, j < N);
    if (j == 1) {                            // r2 = p_1 - grad g(x_0) (g with the cost sign)
      if constexpr (sizeof(T) == 4 && kkt_in_iter_type<F>::value) {
        // in FP32 like the node's terms, W^2 and c staged as floats (gsh): FP64
        // here ran on one lane per point at the 1/64-rate pipe
        float rf = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float e = fabsf(p[k] - float(sgn) * gsh[k] * (xl[k] - gsh[D + k]));
          rf = (e > rf || e != e) ? e : rf;
        }
        r = max_nan(r, (double)rf);
      } else {
#pragma unroll
        for (int k = 0; k < D; ++k)
          r = max_nan(r, fabs((double)p[k] - sgn * a.W2[k] * ((double)xl[k] - a.c[k])));
      }
    }
    return r;
  }
}

template <typename T, class F, int D>
__global__ void __launch_bounds__(256)
kkt_node_kernel(const SolveArgs<T> a, const T* __restrict__ X, const T* __restrict__ P,
                double* __restrict__ kkt) {
  typename F::Shared unused;                 // the node residual reads no family data
  const F fam(a, unused);
  __shared__ T gsh[2 * D];                   // W^2 and c in the iterate type
  for (int k = threadIdx.x; k < D; k += blockDim.x) { gsh[k] = T(a.W2[k]); gsh[D + k] = T(a.c[k]); }
  __syncthreads();
  const int N = a.N;
  const int64_t total = a.B * (int64_t)N;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) - lane;
  const int64_t wstride = (int64_t)gridDim.x * blockDim.x;
  // the whole warp walks the (point, node) list together, so its shuffles see every lane
  for (int64_t base = warp0; base < total; base += wstride) {
    const int64_t idx = base + lane;
    const bool valid = idx < total;
    const int64_t b = valid ? idx / N : -1;
    double r = 0.0;
    if (valid) r = node_residual<T, F, D>(a, fam, X, P, b, 1 + (int)(idx - b * N), gsh);
    unsigned long long v = (unsigned long long)__double_as_longlong(r);
    // maximum over the run of lanes holding the same point (b is nondecreasing in the lane)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long w = __shfl_down_sync(kFull, v, o);
      const long long bw = __shfl_down_sync(kFull, (long long)b, o);
      if (lane + o < 32 && bw == b && w > v) v = w;
    }
    const long long bprev = __shfl_up_sync(kFull, (long long)b, 1);
    if (valid && (lane == 0 || bprev != b))
      atomicMax(reinterpret_cast<unsigned long long*>(kkt + b), v);
  }
}

template <typename T, class F, int D>
hj_status launch_node(const SolveArgs<T>& a, const T* X, const T* P, double* kkt,
                      cudaStream_t s) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HJ_ERR_CUDA;
  if (cudaMemsetAsync(kkt, 0, (size_t)a.B * sizeof(double), s) != cudaSuccess) return HJ_ERR_CUDA;
  const int64_t blocks = (a.B * (int64_t)a.N + 255) / 256;
  const int64_t cap = (int64_t)nsm * 8;
  kkt_node_kernel<T, F, D><<<(int)(blocks < cap ? blocks : cap), 256, 0, s>>>(a, X, P, kkt);
  return cudaGetLastError() == cudaSuccess ? HJ_OK : HJ_ERR_CUDA;
}

}  // namespace

template <typename T>
hj_status launch_kkt_nodes(const hj_problem_s* p, int64_t B, int32_t N, const double* t,
                           const T* X, const T* P, double* kkt, cudaStream_t s) {
  SolveArgs<T> a{};
  a.B = B; a.N = N; a.d = p->d; a.t = t;
  a.W2 = p->W2; a.c = p->c; a.A64 = p->Ad;
  a.qc_m = p->qc[0]; a.qc_ah = p->qc[1]; a.qc_gz = p->qc[2]; a.qc_eps = p->qc[3];
  a.eik_c0 = p->eik[1]; a.eik_c1 = p->eik[2]; a.eik_c2 = p->eik[3];
  fill_family_consts(a);
  a.xb64 = p->xbd; a.vb64 = p->vbd;
  a.cost_sign = (p->family == HJ_FAMILY_EIKONAL && p->eik[0] < 0) ? -1.0 : 1.0;
  switch (p->family) {
    case HJ_FAMILY_QUADRATIC:
      switch (p->d) {
        case 1: return launch_node<T, FamQuadratic<T, 1>, 1>(a, X, P, kkt, s);
        case 2: return launch_node<T, FamQuadratic<T, 2>, 2>(a, X, P, kkt, s);
        case 3: return launch_node<T, FamQuadratic<T, 3>, 3>(a, X, P, kkt, s);
        case 4: return launch_node<T, FamQuadratic<T, 4>, 4>(a, X, P, kkt, s);
        default: return HJ_ERR_UNSUPPORTED;
      }
    case HJ_FAMILY_QUADCOPTER:
      return p->d == 12 ? launch_node<T, FamQuadcopter<T, 12>, 12>(a, X, P, kkt, s)
                        : HJ_ERR_UNSUPPORTED;
    case HJ_FAMILY_TANH_DRIFT:
      if (p->d == 2) return launch_node<T, FamTanhDrift<T, 2>, 2>(a, X, P, kkt, s);
      if (p->d == 4) return launch_node<T, FamTanhDrift<T, 4>, 4>(a, X, P, kkt, s);
      return HJ_ERR_UNSUPPORTED;
    case HJ_FAMILY_EIKONAL:
      if (p->eik_moving) {
        if (p->d == 2) return launch_node<T, FamEikonalMoving<T, 2>, 2>(a, X, P, kkt, s);
        if (p->d == 10) return launch_node<T, FamEikonalMoving<T, 10>, 10>(a, X, P, kkt, s);
      } else {
        if (p->d == 2) return launch_node<T, FamEikonal<T, 2>, 2>(a, X, P, kkt, s);
        if (p->d == 10) return launch_node<T, FamEikonal<T, 10>, 10>(a, X, P, kkt, s);
      }
      return HJ_ERR_UNSUPPORTED;
    default:
      return HJ_ERR_UNSUPPORTED;
  }
}

template hj_status launch_kkt_nodes<float>(const hj_problem_s*, int64_t, int32_t, const double*,
                                           const float*, const float*, double*, cudaStream_t);
template hj_status launch_kkt_nodes<double>(const hj_problem_s*, int64_t, int32_t, const double*,
                                            const double*, const double*, double*, cudaStream_t);

}  // namespace hj
