// Register-resident batched PDHG for the Lax saddle problem (Algorithm 1).
//
// A group of G warps solves one query point at a time.  Lane gl (0..32G-1)
// of the group owns the time nodes j = 1 + gl*NPL .. gl*NPL + NPL (those <= N),
// with x_j, p_j and the relaxed z_j in registers; lane 0 also owns node 0
// (x_0, the g-prox node).  The nearest-neighbour terms of the difference
// operator D ((Dz)_j = z_j - z_{j-1}, (D^T p)_j = p_j - p_{j+1}, Appendix A.1)
// cross a lane boundary once per direction and iteration as warp shuffles, and
// a warp boundary (G > 1) through a shared-memory slot between two barriers.
// Groups draw points from a work counter until the batch is exhausted
// (persistent grid sized to the SM count).
//
// One iteration, per owned node (Section 5.3 updates, loop of Algorithm A.1):
//   ctx  <- H quantities at x_j^k
//   p_j  <- prox_{sigma delta H(x_j^k, .)}(p_j + sigma (z_j - z_{j-1}))     j = 1..N
//   x_0  <- prox_{tau g}(x_0 + tau p_1)
//   x_j  <- x_j - tau (p_j - p_{j+1}) + tau delta grad_x H(x_j^k, p_j)      j = 1..N-1
//   z_j  <- x_j^{k+1} + theta (x_j^{k+1} - x_j^k)
// and, on test iterations, the squared increments summed in FP64 over the group.
#pragma once
#include <cuda_runtime.h>

#include "families.cuh"
#include "hj_internal.cuh"

namespace hj {

constexpr int kWarpsPerCtaG1 = 4;   // independent single-warp groups per CTA when G = 1

template <int G>
constexpr int warp_block_threads() { return (G == 1 ? kWarpsPerCtaG1 : G) * 32; }

// Per-CTA shared memory: the family's data, the g-prox of x_0
// (x_0 <- (v + tau W^2 c) / (1 + tau W^2) as offset and reciprocal), and for
// G > 1 the warp-boundary slots and reduction scratch of the CTA's one group.
template <typename T, class F, int D, int G>
struct WarpShared {
  typename F::Shared fam;
  T g_off[D], g_inv[D];
  double w2d[D], cd[D];
  T zb[G][D];          // z (then x) of each warp's last lane
  T pb[G][D];          // p of each warp's first lane
  double red[G][2];
  double vred[G];
  unsigned long long item;
};

template <int G>
__device__ __forceinline__ void group_sync() {
  if constexpr (G > 1) __syncthreads();
}

template <typename T, class F, int D, int NPL, int G>
__device__ __forceinline__ void solve_point(const SolveArgs<T>& a, const F& fam, int64_t item,
                                            int lane, int wg, WarpShared<T, F, D, G>& sh) {
  const PointRef<T> pt = point_ref(a, item);
  const int N = pt.N;
  const int gl = wg * 32 + lane;
  if (N < 1 || N > 32 * G * NPL) {          // the host never routes such a point here
    if (gl == 0) { a.status[pt.id] = HJ_POINT_INVALID; a.iters[pt.id] = 0; a.V[pt.id] = 0.0; }
    return;
  }
  // iteration constants in the iterate type only (delta = t / N)
  const T sig = a.sigma_t, tau = a.tau_t, th = a.theta_t;
  const T delta_t = T(a.t[pt.id]) / T(N);
  const T lam = sig * delta_t, taud = tau * delta_t;
  const typename F::PC pc = fam.point(lam);
  const uint64_t gid = (uint64_t)(a.point_offset + pt.id);

  T x[NPL][D], p[NPL][D], z[NPL][D];
  T x0[D], z0[D];
  const int jbase = 1 + gl * NPL;
  {
    double xqd[D];
#pragma unroll
    for (int k = 0; k < D; ++k) xqd[k] = pt.xq[k];
    if (a.warm_x == nullptr) {
#pragma unroll
      for (int i = 0; i < NPL; ++i) {
        const int j = jbase + i;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          T xv = T(0), pv = T(0);
          if (j < N) xv = T(xqd[k] + a.radius * uniform_pm1(a.seed, gid, 0, j, k));
          else if (j == N) xv = T(xqd[k]);
          if (j <= N) pv = T(a.radius * uniform_pm1(a.seed, gid, 1, j, k));
          x[i][k] = xv; p[i][k] = pv; z[i][k] = xv;
        }
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        x0[k] = T(xqd[k] + a.radius * uniform_pm1(a.seed, gid, 0, 0, k));
        z0[k] = x0[k];
      }
    } else {
      const T* wx = a.warm_x + pt.traj;
      const T* wp = a.warm_p + pt.traj;
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
  }
  if constexpr (G > 1) {
    if (lane == 31)
#pragma unroll
      for (int k = 0; k < D; ++k) sh.zb[wg][k] = z[NPL - 1][k];
  }

  int k_it = 0;
  int8_t st = HJ_POINT_MAX_ITER;
  const int max_iter = a.max_iter, check_every = a.check_every;
  int until_check = check_every;
  while (k_it < max_iter) {
    ++k_it;
    const bool chk = (--until_check == 0) || (k_it == max_iter);
    if (until_check == 0) until_check = check_every;
    T rx = T(0), rp = T(0);
    typename F::Ctx ctx[NPL];
    group_sync<G>();                                            // zb of the last iteration
    // ---- dual step, nodes 1..N (z_{j-1} of the first owned node from the left lane)
    T zl[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const T up = __shfl_up_sync(kFull, z[NPL - 1][k], 1);
      T v = up;
      if (lane == 0) {
        if constexpr (G > 1) v = (wg == 0) ? z0[k] : sh.zb[wg - 1][k];
        else v = z0[k];
      }
      zl[k] = v;
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
        fam.prox(ctx[i], pc, x[i], v);
        if (chk) {
#pragma unroll
          for (int k = 0; k < D; ++k) { const T e = v[k] - p[i][k]; rp += e * e; }
        }
#pragma unroll
        for (int k = 0; k < D; ++k) p[i][k] = v[k];
      }
    }
    // ---- primal step: p_{j+1} of the last owned node from the right lane
    if constexpr (G > 1) {
      if (lane == 0)
#pragma unroll
        for (int k = 0; k < D; ++k) sh.pb[wg][k] = p[0][k];
    }
    group_sync<G>();
    T pr[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      T v = __shfl_down_sync(kFull, p[0][k], 1);
      if constexpr (G > 1) {
        if (lane == 31 && wg + 1 < G) v = sh.pb[wg + 1][k];
      }
      pr[k] = v;
    }
    if (gl == 0) {
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
    if constexpr (G > 1) {
      if (lane == 31)
#pragma unroll
        for (int k = 0; k < D; ++k) sh.zb[wg][k] = z[NPL - 1][k];
    }
    if (chk) {
      // lane partials summed across the warp in the iterate type, then in FP64
      double sx = (double)warp_sum<T>(rx);
      double sp = (double)warp_sum<T>(rp);
      if constexpr (G > 1) {
        if (lane == 0) { sh.red[wg][0] = sx; sh.red[wg][1] = sp; }
        __syncthreads();
        sx = 0.0; sp = 0.0;
#pragma unroll
        for (int w = 0; w < G; ++w) { sx += sh.red[w][0]; sp += sh.red[w][1]; }
      }
      if (!(isfinite(sx) && isfinite(sp))) { st = HJ_POINT_NONFINITE; break; }
      if (sx < a.tol && sp < a.tol) { st = HJ_POINT_CONVERGED; break; }
    }
  }

  // ---- value (fval of Algorithm 1) in FP64, and outputs
  if constexpr (G > 1) {
    if (lane == 31)
#pragma unroll
      for (int k = 0; k < D; ++k) sh.zb[wg][k] = x[NPL - 1][k];
    __syncthreads();
  }
  double acc = 0.0;
  {
    const double delta = a.t[pt.id] / N;
    T xl[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const T up = __shfl_up_sync(kFull, x[NPL - 1][k], 1);
      T v = up;
      if (lane == 0) {
        if constexpr (G > 1) v = (wg == 0) ? x0[k] : sh.zb[wg - 1][k];
        else v = x0[k];
      }
      xl[k] = v;
    }
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
      if (jbase + i <= N) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const double xm = (double)((i == 0) ? xl[k] : x[i - 1][k]);
          s += (double)p[i][k] * ((double)x[i][k] - xm);
        }
        acc += s - delta * fam.H64(x[i], p[i]);
      }
    }
    if (gl == 0) {
      double g = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double e = (double)x0[k] - sh.cd[k];
        g += sh.w2d[k] * e * e;
      }
      acc += 0.5 * g;
    }
  }
  acc = warp_sum<double>(acc);
  if constexpr (G > 1) {
    if (lane == 0) sh.vred[wg] = acc;
    __syncthreads();
    acc = 0.0;
#pragma unroll
    for (int w = 0; w < G; ++w) acc += sh.vred[w];
  }
  if (gl == 0) {
    a.V[pt.id] = acc;
    a.iters[pt.id] = k_it;
    a.status[pt.id] = st;
  }
  if (a.traj_x != nullptr) {
    T* o = a.traj_x + pt.traj;
#pragma unroll
    for (int i = 0; i < NPL; ++i)
      if (jbase + i <= N)
#pragma unroll
        for (int k = 0; k < D; ++k) o[(size_t)(jbase + i) * D + k] = x[i][k];
    if (gl == 0)
#pragma unroll
      for (int k = 0; k < D; ++k) o[k] = x0[k];
  }
  if (a.traj_p != nullptr) {
    T* o = a.traj_p + pt.traj;
#pragma unroll
    for (int i = 0; i < NPL; ++i)
      if (jbase + i <= N)
#pragma unroll
        for (int k = 0; k < D; ++k) o[(size_t)(jbase + i) * D + k] = p[i][k];
    if (gl == 0)
#pragma unroll
      for (int k = 0; k < D; ++k) o[k] = T(0);
  }
}

template <typename T, class F, int D, int NPL, int G>
__global__ void __launch_bounds__(warp_block_threads<G>())
lax_warp_kernel(const SolveArgs<T> a) {
  __shared__ WarpShared<T, F, D, G> sh;
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
  const int wg = (G == 1) ? 0 : (int)(threadIdx.x >> 5);
  for (;;) {
    int64_t item;
    if constexpr (G == 1) {
      unsigned long long bb = 0;
      if (lane == 0) bb = atomicAdd(a.counter, 1ull);
      item = (int64_t)__shfl_sync(kFull, bb, 0);
    } else {
      __syncthreads();                       // the previous point is finished by every warp
      if (threadIdx.x == 0) sh.item = atomicAdd(a.counter, 1ull);
      __syncthreads();
      item = (int64_t)sh.item;
    }
    if (item >= a.B) break;
    solve_point<T, F, D, NPL, G>(a, fam, item, lane, wg, sh);
  }
}

template <typename T, class F, int D, int NPL, int G>
hj_status launch_warp_cfg(const SolveArgs<T>& a, cudaStream_t s) {
  static int blocks_per_sm = -1;
  static int num_sms = 0;
  auto kern = lax_warp_kernel<T, F, D, NPL, G>;
  constexpr int threads = warp_block_threads<G>();
  if (blocks_per_sm < 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HJ_ERR_CUDA;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return HJ_ERR_CUDA;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, threads, 0) != cudaSuccess)
      return HJ_ERR_CUDA;
    blocks_per_sm = bps > 0 ? bps : 1;
  }
  constexpr int points_per_cta = (G == 1) ? kWarpsPerCtaG1 : 1;
  const int64_t need = (a.B + points_per_cta - 1) / points_per_cta;
  const int64_t cap = (int64_t)blocks_per_sm * num_sms;
  const int grid = (int)(need < cap ? need : cap);
  if (grid <= 0) return HJ_OK;
  kern<<<grid, threads, 0, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? HJ_OK : HJ_ERR_CUDA;
}

// Every (G, NPL) the library instantiates: FP32 G in {1,2,4,8} x NPL in {1,2};
// FP64 G in {1,2,4,8} x NPL = 1.
template <typename T, template <typename, int> class F, int D>
hj_status launch_warp_shape(const SolveArgs<T>& a, WarpConfig c, cudaStream_t s) {
  constexpr bool f64 = sizeof(T) == 8;
  if (c.NPL == 1) {
    switch (c.G) {
      case 1: return launch_warp_cfg<T, F<T, D>, D, 1, 1>(a, s);
      case 2: return launch_warp_cfg<T, F<T, D>, D, 1, 2>(a, s);
      case 4: return launch_warp_cfg<T, F<T, D>, D, 1, 4>(a, s);
      case 8: return launch_warp_cfg<T, F<T, D>, D, 1, 8>(a, s);
      default: return HJ_ERR_UNSUPPORTED;
    }
  }
  if constexpr (!f64) {
    if (c.NPL == 2) {
      switch (c.G) {
        case 1: return launch_warp_cfg<T, F<T, D>, D, 2, 1>(a, s);
        case 2: return launch_warp_cfg<T, F<T, D>, D, 2, 2>(a, s);
        case 4: return launch_warp_cfg<T, F<T, D>, D, 2, 4>(a, s);
        case 8: return launch_warp_cfg<T, F<T, D>, D, 2, 8>(a, s);
        default: return HJ_ERR_UNSUPPORTED;
      }
    }
  }
  return HJ_ERR_UNSUPPORTED;
}

}  // namespace hj
