// Register-resident batched PDHG for the Lax saddle problem (Algorithm 1).
//
// One warp solves one query point at a time.  Lane l owns the time nodes
// j = 1 + l*NPL .. l*NPL + NPL (those <= N), with x_j, p_j and the relaxed
// z_j in registers; lane 0 also owns node 0 (x_0, the g-prox node).  The
// nearest-neighbour terms of the difference operator D ((Dz)_j = z_j - z_{j-1},
// (D^T p)_j = p_j - p_{j+1}, Appendix A.1) cross a lane boundary once per
// iteration each, as warp shuffles.  Warps draw points from a work counter
// until the batch is exhausted (persistent grid sized to the SM count).
//
// One iteration, per owned node (Section 5.3 updates, loop of Algorithm A.1):
//   ctx  <- H quantities at x_j^k
//   p_j  <- prox_{sigma delta H(x_j^k, .)}(p_j + sigma (z_j - z_{j-1}))     j = 1..N
//   x_0  <- prox_{tau g}(x_0 + tau p_1)
//   x_j  <- x_j - tau (p_j - p_{j+1}) + tau delta grad_x H(x_j^k, p_j)      j = 1..N-1
//   z_j  <- x_j^{k+1} + theta (x_j^{k+1} - x_j^k)
// and, on test iterations, the squared increments summed in FP64 across the warp.
#include <cuda_runtime.h>

#include "families.cuh"
#include "hj_internal.cuh"

namespace hj {

constexpr int kWarpsPerCta = 4;

// Per-CTA constants in shared memory (kept out of registers): the family's own
// data and the g-prox of x_0, x_0 <- (v + tau W^2 c) / (1 + tau W^2), as an
// offset and a reciprocal per coordinate.
template <typename T, class F, int D>
struct WarpShared {
  typename F::Shared fam;
  T g_off[D], g_inv[D];
  double w2d[D], cd[D];
};

template <typename T, class F, int D, int NPL>
__device__ __forceinline__ void solve_point(const SolveArgs<T>& a, const F& fam, int64_t b,
                                            int lane, const WarpShared<T, F, D>& sh) {
  const int N = a.N;
  const double tb = a.t[b];
  const double delta = tb / N;
  const T sig = T(a.sigma), tau = T(a.tau), th = T(a.theta);
  const T lam = T(a.sigma * delta), taud = T(a.tau * delta);
  const uint64_t pt = (uint64_t)(a.point_offset + b);

  double xqd[D];
#pragma unroll
  for (int k = 0; k < D; ++k) xqd[k] = a.xq[b * D + k];

  T x[NPL][D], p[NPL][D], z[NPL][D];
  T x0[D], z0[D];
  const int jbase = 1 + lane * NPL;
  const size_t stride = (size_t)(N + 1) * D;
  if (a.warm_x == nullptr) {
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
      const int j = jbase + i;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        T xv = T(0), pv = T(0);
        if (j < N) xv = T(xqd[k] + a.radius * uniform_pm1(a.seed, pt, 0, j, k));
        else if (j == N) xv = T(xqd[k]);
        if (j <= N) pv = T(a.radius * uniform_pm1(a.seed, pt, 1, j, k));
        x[i][k] = xv; p[i][k] = pv; z[i][k] = xv;
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      x0[k] = T(xqd[k] + a.radius * uniform_pm1(a.seed, pt, 0, 0, k));
      z0[k] = x0[k];
    }
  } else {
    const T* wx = a.warm_x + b * stride;
    const T* wp = a.warm_p + b * stride;
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
      const int j = jbase + i;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        T xv = T(0), pv = T(0);
        if (j < N) xv = wx[(size_t)j * D + k];
        else if (j == N) xv = T(xqd[k]);
        if (j <= N) pv = wp[(size_t)j * D + k];
        x[i][k] = xv; p[i][k] = pv; z[i][k] = xv;
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) { x0[k] = wx[k]; z0[k] = x0[k]; }
  }

  int k_it = 0;
  int8_t st = HJ_POINT_MAX_ITER;
  const int max_iter = a.max_iter, check_every = a.check_every;
  while (k_it < max_iter) {
    ++k_it;
    const bool chk = (k_it % check_every == 0) || (k_it == max_iter);
    T rx = T(0), rp = T(0);
    typename F::Ctx ctx[NPL];
    // ---- dual step, nodes 1..N (z_{j-1} of the first owned node comes from the left lane)
    T zl[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const T up = __shfl_up_sync(kFull, z[NPL - 1][k], 1);
      zl[k] = (lane == 0) ? z0[k] : up;
    }
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
      if (jbase + i <= N) {
        fam.context(x[i], ctx[i]);
        T v[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const T zm = (i == 0) ? zl[k] : z[i - 1][k];
          v[k] = p[i][k] + sig * (z[i][k] - zm);
        }
        fam.prox(ctx[i], x[i], v, lam);
        if (chk) {
#pragma unroll
          for (int k = 0; k < D; ++k) { const T e = v[k] - p[i][k]; rp += e * e; }
        }
#pragma unroll
        for (int k = 0; k < D; ++k) p[i][k] = v[k];
      }
    }
    // ---- primal step: p_{j+1} of the last owned node comes from the right lane
    T pr[D];
#pragma unroll
    for (int k = 0; k < D; ++k) pr[k] = __shfl_down_sync(kFull, p[0][k], 1);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const T vx = x0[k] + tau * p[0][k];                  // (D^T p)_0 = -p_1
        const T xn = (vx + sh.g_off[k]) * sh.g_inv[k];
        if (chk) { const T e = xn - x0[k]; rx += e * e; }
        z0[k] = xn + th * (xn - x0[k]);
        x0[k] = xn;
      }
    }
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
      if (jbase + i < N) {
        T xn[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const T pn = (i == NPL - 1) ? pr[k] : p[i + 1][k];
          xn[k] = x[i][k] - tau * (p[i][k] - pn);
        }
        if (F::kHasGradX) {
          T g[D];
          fam.gradx(ctx[i], x[i], p[i], g);
          T base[D];
#pragma unroll
          for (int k = 0; k < D; ++k) { base[k] = xn[k]; xn[k] = base[k] + taud * g[k]; }
          for (int s = 1; s < a.inner_steps; ++s) {
            typename F::Ctx c2;
            fam.context(xn, c2);
            fam.gradx(c2, xn, p[i], g);
#pragma unroll
            for (int k = 0; k < D; ++k) xn[k] = base[k] + taud * g[k];
          }
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
          if (chk) { const T e = xn[k] - x[i][k]; rx += e * e; }
          z[i][k] = xn[k] + th * (xn[k] - x[i][k]);
          x[i][k] = xn[k];
        }
      }
    }
    if (chk) {
      const double sx = warp_sum((double)rx);
      const double sp = warp_sum((double)rp);
      if (!(isfinite(sx) && isfinite(sp))) { st = HJ_POINT_NONFINITE; break; }
      if (sx < a.tol && sp < a.tol) { st = HJ_POINT_CONVERGED; break; }
    }
  }

  // ---- value (fval of Algorithm 1) in FP64, and outputs
  double acc = 0.0;
  {
    double xl[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const T up = __shfl_up_sync(kFull, x[NPL - 1][k], 1);
      xl[k] = (double)((lane == 0) ? x0[k] : up);
    }
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
      if (jbase + i <= N) {
        double xd[D], pd[D];
#pragma unroll
        for (int k = 0; k < D; ++k) { xd[k] = (double)x[i][k]; pd[k] = (double)p[i][k]; }
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const double xm = (i == 0) ? xl[k] : (double)x[i - 1][k];
          s += pd[k] * (xd[k] - xm);
        }
        acc += s - delta * fam.H64(xd, pd);
      }
    }
    if (lane == 0) {
      double g = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double e = (double)x0[k] - sh.cd[k];
        g += sh.w2d[k] * e * e;
      }
      acc += 0.5 * g;
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) {
    a.V[b] = acc;
    a.iters[b] = k_it;
    a.status[b] = st;
  }
  if (a.traj_x != nullptr) {
    T* o = a.traj_x + b * stride;
#pragma unroll
    for (int i = 0; i < NPL; ++i)
      if (jbase + i <= N)
#pragma unroll
        for (int k = 0; k < D; ++k) o[(size_t)(jbase + i) * D + k] = x[i][k];
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < D; ++k) o[k] = x0[k];
  }
  if (a.traj_p != nullptr) {
    T* o = a.traj_p + b * stride;
#pragma unroll
    for (int i = 0; i < NPL; ++i)
      if (jbase + i <= N)
#pragma unroll
        for (int k = 0; k < D; ++k) o[(size_t)(jbase + i) * D + k] = p[i][k];
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < D; ++k) o[k] = T(0);
  }
}

template <typename T, class F, int D, int NPL>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
lax_warp_kernel(const SolveArgs<T> a) {
  __shared__ WarpShared<T, F, D> sh;
  F::load_shared(a, sh.fam);
  for (int k = threadIdx.x; k < D; k += blockDim.x) {
    const double w2 = a.W2[k], c = a.c[k];
    sh.w2d[k] = w2;
    sh.cd[k] = c;
    sh.g_off[k] = T(a.tau * w2 * c);
    sh.g_inv[k] = T(1.0 / (1.0 + a.tau * w2));
  }
  __syncthreads();
  const F fam(a, sh.fam);
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long bb = 0;
    if (lane == 0) bb = atomicAdd(a.counter, 1ull);
    bb = __shfl_sync(kFull, bb, 0);
    if ((int64_t)bb >= a.B) break;
    solve_point<T, F, D, NPL>(a, fam, (int64_t)bb, lane, sh);
  }
}

template <typename T, class F, int D, int NPL>
static hj_status launch_one(const SolveArgs<T>& a, cudaStream_t s) {
  static int blocks_per_sm = -1;
  static int num_sms = 0;
  auto kern = lax_warp_kernel<T, F, D, NPL>;
  if (blocks_per_sm < 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HJ_ERR_CUDA;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return HJ_ERR_CUDA;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kWarpsPerCta * 32, 0) !=
        cudaSuccess)
      return HJ_ERR_CUDA;
    blocks_per_sm = bps > 0 ? bps : 1;
  }
  const int64_t need = (a.B + kWarpsPerCta - 1) / kWarpsPerCta;
  const int64_t cap = (int64_t)blocks_per_sm * num_sms;
  const int grid = (int)(need < cap ? need : cap);
  kern<<<grid, kWarpsPerCta * 32, 0, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? HJ_OK : HJ_ERR_CUDA;
}

template <typename T, template <typename, int> class F, int D>
static hj_status dispatch_npl(const SolveArgs<T>& a, cudaStream_t s) {
  if (a.N <= 32) return launch_one<T, F<T, D>, D, 1>(a, s);
  if (a.N <= 64) return launch_one<T, F<T, D>, D, 2>(a, s);
  if constexpr (D <= 4) {
    if (a.N <= 128) return launch_one<T, F<T, D>, D, 4>(a, s);
  }
  return HJ_ERR_UNSUPPORTED;
}

template <typename T>
hj_status launch_warp_solver(int family, const SolveArgs<T>& a, cudaStream_t s) {
  switch (family) {
    case HJ_FAMILY_QUADRATIC:
      switch (a.d) {
        case 1: return dispatch_npl<T, FamQuadratic, 1>(a, s);
        case 2: return dispatch_npl<T, FamQuadratic, 2>(a, s);
        case 3: return dispatch_npl<T, FamQuadratic, 3>(a, s);
        case 4: return dispatch_npl<T, FamQuadratic, 4>(a, s);
        case 8: return dispatch_npl<T, FamQuadratic, 8>(a, s);
        default: return HJ_ERR_UNSUPPORTED;
      }
    case HJ_FAMILY_QUADCOPTER:
      if (a.d != 12) return HJ_ERR_UNSUPPORTED;
      return dispatch_npl<T, FamQuadcopter, 12>(a, s);
    case HJ_FAMILY_TANH_DRIFT:
      switch (a.d) {
        case 2: return dispatch_npl<T, FamTanhDrift, 2>(a, s);
        case 4: return dispatch_npl<T, FamTanhDrift, 4>(a, s);
        case 8: return dispatch_npl<T, FamTanhDrift, 8>(a, s);
        default: return HJ_ERR_UNSUPPORTED;
      }
    default:
      return HJ_ERR_UNSUPPORTED;
  }
}

template hj_status launch_warp_solver<float>(int, const SolveArgs<float>&, cudaStream_t);
template hj_status launch_warp_solver<double>(int, const SolveArgs<double>&, cudaStream_t);

}  // namespace hj
