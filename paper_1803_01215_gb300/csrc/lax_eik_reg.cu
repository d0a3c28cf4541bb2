// Coordinate-parallel batched PDHG for the eikonal family with the state in
// registers (Section 6.1: H = c(x)|p|_2, c(x) = c0 + c1 exp(-c2 |x - x_b|^2),
// Algorithm 1 with the shrink_2 dual step and one gradient step in x), static
// bump, backward Euler, N <= 16, d up to 2048 (a cluster of two CTAs above
// 1024): the paper's dimensional-scaling runs (N = 10) up to d = 2000.
//
// One CTA solves one query point.  Thread t owns the coordinates
// k = t + c T (c < CPT) and keeps x_j, p_j, z_j of every node j = 0..N of those
// coordinates in registers for the whole solve (N <= NM, the loops over nodes
// unrolled), so the difference operator never leaves the thread and the
// iteration touches shared memory only for the node scalars.  Per iteration:
//   1. the node scalars |x_j - x_b|^2 and |v_j|^2 (v_j = p_j + sigma (z_j - z_{j-1}))
//      of the previous pass, summed over the warps: thread j - 1 forms node j's
//      shrink factor and x-step coefficient tau delta |p_j| (-2 c1 c2 e_j);
//      barrier;
//   2. each thread, per coordinate: the dual step of every node (old z), the
//      g-prox of x_0, the x-steps of nodes 1..N-1 and the relaxation, then its
//      parts of the next iteration's 2N node scalars, which the warp sums by
//      one reduce-scatter (each lane keeps half of its values and sends the
//      other half at each of five exchange steps: sum_s ceil(m_s / 2)
//      shuffles for 2N values instead of 10 N) and parks in shared memory;
//      barrier.
// The test iterations add the squared increments: per-thread partials in the
// iterate type, reduced over the warp in that type, accumulated over the warps
// as double-floats (FP32 iterates: as accurate as FP64, on the FP32 pipe) or in
// FP64 (stop_verdict).  The negative equation (cost_sign = -1) runs the
// positive one with -g and returns -V and -p, as in Section 6.1.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "hj_internal.cuh"

namespace cg = cooperative_groups;

namespace hj {

namespace {

constexpr int kRegMaxThreads = 512;
constexpr int kRegMaxWarps = kRegMaxThreads / 32;

template <typename T>
__device__ __forceinline__ T expr(T y) { return exp(y); }
template <>
__device__ __forceinline__ float expr<float>(float y) { return __expf(y); }

template <typename T>
__device__ __forceinline__ T sqrtr(T y) { return sqrt(y); }
template <>
__device__ __forceinline__ float sqrtr<float>(float y) { return sqrtf(y); }

// one exchange step of warp_reduce_scatter on the first m values (then the next)
template <int S, int m, typename T, int M>
__device__ __forceinline__ void rs_step(T (&v)[M], int lane, int& base, int& cnt) {
  if constexpr (S < 5) {
    constexpr int o = 16 >> S;
    constexpr int h = (m + 1) / 2;
    const bool b = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const T lo = v[i];
      T hi = T(0);
      if (i + h < m) hi = v[i + h < m ? i + h : 0];
      const T keep = b ? hi : lo;
      v[i] = keep + __shfl_xor_sync(kFull, b ? lo : hi, o);
    }
    if (b) { base += h; cnt -= h; } else { cnt = cnt < h ? cnt : h; }
    rs_step<S + 1, h>(v, lane, base, cnt);
  }
}

// Sum each of M per-lane values over the 32 lanes of the warp.  At exchange
// step s (lane offset o = 16 >> s) a lane keeps one half of its current range
// of values (the lower half if its bit o is clear) and sends the other half to
// lane ^ o, adding what it receives; after five steps each lane holds the warp
// total of one value, `idx`, valid when it returns true (every value lands on
// exactly one lane).  Ranges are padded to the half size with zeros.
template <typename T, int M>
__device__ __forceinline__ bool warp_reduce_scatter(T (&v)[M], int lane, T& out, int& idx) {
  static_assert(M >= 1 && M <= 32, "at most one value per lane");
  int base = 0, cnt = M;
  rs_step<0, M>(v, lane, base, cnt);
  out = v[0];
  idx = base;
  return cnt >= 1;
}

// barrier of the CTA, or of the cluster (with release / acquire of shared memory)
template <int CL>
__device__ __forceinline__ void csync() {
  if constexpr (CL > 1) cg::this_cluster().sync();
  else __syncthreads();
}

// CL = 2: a cluster of two CTAs solves each point, CTA r owning the coordinates
// r T CPT + (t + c T); every barrier of the iteration is then a cluster
// barrier, the node sums are double-buffered (the other CTA reads them through
// distributed shared memory while this one fills the next buffer), and both
// CTAs form the node scalars from both CTAs' sums.
template <typename T, int CPT, int NM, bool EXACT, int CL>
__global__ void __launch_bounds__(kRegMaxThreads) lax_eik_reg_kernel(const SolveArgs<T> a) {
  constexpr int NB = CL > 1 ? 2 : 1;
  __shared__ T red[NB][kRegMaxWarps][2 * NM];    // per-warp node sums: |x_j - x_b|^2, |v_j|^2
  __shared__ T keep_s[NM + 1], coef_s[NM + 1];
  __shared__ T tred[kRegMaxWarps][2];              // per-warp stopping sums
  __shared__ double vred[kRegMaxWarps];
  __shared__ unsigned long long s_point;
  const int d = a.d;
  const int T_ = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = T_ >> 5;
  unsigned rank = 0;
  const T* peer_red = nullptr;                     // the other CTA's red, tred, vred, s_point
  const T* peer_tred = nullptr;
  const double* peer_vred = nullptr;
  const unsigned long long* peer_point = nullptr;
  if constexpr (CL > 1) {
    cg::cluster_group cl = cg::this_cluster();
    rank = cl.block_rank();
    peer_red = cl.map_shared_rank(&red[0][0][0], rank ^ 1u);
    peer_tred = cl.map_shared_rank(&tred[0][0], rank ^ 1u);
    peer_vred = cl.map_shared_rank(&vred[0], rank ^ 1u);
    peer_point = cl.map_shared_rank(&s_point, 0u);
  }
  const T sig = a.sigma_t, tau = a.tau_t, th = a.theta_t;
  const T c0 = a.eik_t[0], c1 = a.eik_t[1], c2 = a.eik_t[2];
  const int kbase = (int)rank * T_ * CPT;          // first coordinate of this CTA's span
  // the thread's coordinates: bump centre and the g-prox (with the cost sign)
  bool own[CPT];
  T xbk[CPT], goff[CPT], ginv[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    const int k = kbase + tid + c * T_;
    own[c] = k < d;
    const double w2 = own[c] ? a.cost_sign * a.W2[k] : 0.0, cc = own[c] ? a.c[k] : 0.0;
    xbk[c] = own[c] ? a.xb[k] : T(0);
    goff[c] = T(a.tau * w2 * cc);
    ginv[c] = T(1.0 / (1.0 + a.tau * w2));
  }

  for (;;) {
    csync<CL>();                                  // the previous point is done in every CTA
    if (tid == 0 && rank == 0) s_point = draw_item(a);
    csync<CL>();
    const int64_t item = (int64_t)(CL > 1 ? *peer_point : s_point);
    if (item >= a.B) break;
    const PointRef<T> ref = point_ref(a, item);
    const int64_t b = ref.id;
    // EXACT: every point has N = NM (a uniform batch), so the node guards fold away
    const int N = EXACT ? NM : ref.N;
    if (ref.N != N || N < 1 || N > NM) {          // the host never routes such a point here
      if (tid == 0 && rank == 0) { a.status[b] = HJ_POINT_INVALID; a.iters[b] = 0; a.V[b] = 0.0; }
      continue;
    }
    const T delta_t = T(a.t[b]) / T(N);
    const T lam = sig * delta_t, taud = tau * delta_t;
    const uint64_t pt = (uint64_t)(a.point_offset + b);

    // ---- initial iterate (Section 6 random guess, or a warm start), in registers
    T x[CPT][NM + 1], p[CPT][NM + 1], z[CPT][NM + 1];
    {
      const InitGuess<T> ig(a.radius);
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int k = kbase + tid + c * T_;
        const double xq = own[c] ? ref.xq[k] : 0.0;
#pragma unroll
        for (int j = 0; j <= NM; ++j) {
          T xv = T(0), pv = T(0);
          if (own[c] && j <= N) {
            if (a.warm_x == nullptr) {
              xv = (j < N) ? ig.x(xq, a.seed, pt, j, k) : T(xq);
              if (j >= 1) pv = ig.p(a.seed, pt, j, k);
            } else {
              xv = (j < N) ? a.warm_x[ref.traj + (size_t)j * d + k] : T(xq);
              if (j >= 1) pv = T(a.cost_sign) * a.warm_p[ref.traj + (size_t)j * d + k];
            }
          }
          x[c][j] = xv; p[c][j] = pv; z[c][j] = xv;
        }
      }
    }

    int buf = 0;                                  // red buffer being filled (CL = 2)
    // node j's two sums over every warp of the point; for CL = 2 both CTAs add
    // CTA 0's warps, then CTA 1's, so they form bitwise the same node scalars
    auto node_total = [&](int j, T& r2, T& n2) {
      const T* own_b = &red[buf][0][0];
      if constexpr (CL > 1) {
        const T* peer_b = peer_red + (size_t)buf * kRegMaxWarps * 2 * NM;
        const T* r0 = rank == 0 ? own_b : peer_b;
        const T* r1 = rank == 0 ? peer_b : own_b;
        for (int w = 0; w < nwarps; ++w) { r2 += r0[w * 2 * NM + 2 * (j - 1)]; n2 += r0[w * 2 * NM + 2 * (j - 1) + 1]; }
        for (int w = 0; w < nwarps; ++w) { r2 += r1[w * 2 * NM + 2 * (j - 1)]; n2 += r1[w * 2 * NM + 2 * (j - 1) + 1]; }
      } else {
        for (int w = 0; w < nwarps; ++w) { r2 += own_b[w * 2 * NM + 2 * (j - 1)]; n2 += own_b[w * 2 * NM + 2 * (j - 1) + 1]; }
      }
    };
    // this thread's parts of the 2N node scalars at the current iterate
    // (dual = true: |v_j|^2 with v_j = p_j + sigma (z_j - z_{j-1}); else |p_j|^2),
    // summed over the warp and parked in red[buf][warp]
    auto node_sums = [&](bool dual) {
      T s[2 * NM];
#pragma unroll
      for (int j = 1; j <= NM; ++j) {
        T r2 = T(0), v2 = T(0);
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          const T y = x[c][j] - xbk[c];
          r2 += y * y;
          const T v = dual ? p[c][j] + sig * (z[c][j] - z[c][j - 1]) : p[c][j];
          v2 += v * v;
        }
        s[2 * (j - 1)] = (j <= N) ? r2 : T(0);
        s[2 * (j - 1) + 1] = (j <= N) ? v2 : T(0);
      }
      T tot;
      int idx;
      if (warp_reduce_scatter<T, 2 * NM>(s, lane, tot, idx)) red[buf][warp][idx] = tot;
    };

    // one iteration; CHK adds the squared increments (test iterations only)
    auto step = [&](auto chk_tag, T& rx, T& rp) {
      constexpr bool CHK = decltype(chk_tag)::value;
      csync<CL>();                                // red[buf] complete (in every CTA)
      if (tid < N) {                              // node j = tid + 1: shrink and x-step coefficient
        const int j = tid + 1;
        T r2 = T(0), n2 = T(0);
        node_total(j, r2, n2);
        const T e = expr<T>(-c2 * r2);
        const T n = sqrtr<T>(n2), thr = lam * (c0 + c1 * e);
        keep_s[j] = (n > thr) ? (n - thr) / n : T(0);
        coef_s[j] = taud * ((n > thr) ? n - thr : T(0)) * (T(-2) * c1 * c2 * e);
      }
      __syncthreads();                            // keep, coef ready; red free (CL = 1)
      if constexpr (CL > 1) buf ^= 1;             // the next sums go to the other buffer
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        // dual step of every node with the old z
#pragma unroll
        for (int j = NM; j >= 1; --j) {
          if (j <= N) {
            const T pn = keep_s[j] * (p[c][j] + sig * (z[c][j] - z[c][j - 1]));
            if constexpr (CHK) { const T df = pn - p[c][j]; rp += df * df; }
            p[c][j] = pn;
          }
        }
        // x_0: prox of tau g; x_j, j = 1..N-1: gradient step; relaxation
        {
          const T xo = x[c][0];
          const T xn = (xo + tau * p[c][1] + goff[c]) * ginv[c];
          if constexpr (CHK) { const T df = xn - xo; rx += df * df; }
          z[c][0] = xn + th * (xn - xo);
          x[c][0] = xn;
        }
#pragma unroll
        for (int j = 1; j < NM; ++j) {
          if (j < N) {
            const T xo = x[c][j];
            const T xn = xo - tau * (p[c][j] - p[c][j + 1]) + coef_s[j] * (xo - xbk[c]);
            if constexpr (CHK) { const T df = xn - xo; rx += df * df; }
            z[c][j] = xn + th * (xn - xo);
            x[c][j] = xn;
          }
        }
      }
      node_sums(true);                            // the next iteration's node scalars
    };

    int k_it = 0;
    int8_t st = HJ_POINT_MAX_ITER;
    node_sums(true);                              // the first iteration's node scalars
    const int max_iter = a.max_iter, check_every = a.check_every;
    while (k_it < max_iter) {
      // check_every - 1 plain iterations (fewer before max_iter), then a test
      const int left = max_iter - k_it;
      const int plain = (check_every - 1 < left - 1) ? check_every - 1 : left - 1;
      T dx = T(0), dp = T(0);
      for (int r = 0; r < plain; ++r) step(std::integral_constant<bool, false>{}, dx, dp);
      T rx = T(0), rp = T(0);
      step(std::integral_constant<bool, true>{}, rx, rp);
      k_it += plain + 1;
      const T wx = warp_sum<T>(rx), wp = warp_sum<T>(rp);
      if (lane == 0) { tred[warp][0] = wx; tred[warp][1] = wp; }
      csync<CL>();
      // lane w < nwarps: CTA 0's warp w, then CTA 1's warps (CL = 2), the same
      // inputs in the same order in both CTAs, so both take the same verdict
      T vx = T(0), vp = T(0);
      {
        const T* t0 = (CL > 1 && rank != 0) ? peer_tred : &tred[0][0];
        const T* t1 = (CL > 1 && rank == 0) ? peer_tred : &tred[0][0];
        if (lane < nwarps) {
          vx = t0[2 * lane]; vp = t0[2 * lane + 1];
        } else if (CL > 1 && lane < 2 * nwarps) {
          vx = t1[2 * (lane - nwarps)]; vp = t1[2 * (lane - nwarps) + 1];
        }
      }
      const int verdict = stop_verdict_lanes<T>(a, vx, vp);   // 1 converged, 2 non-finite
      if (verdict == 2) { st = HJ_POINT_NONFINITE; break; }
      if (verdict == 1) { st = HJ_POINT_CONVERGED; break; }
    }

    // ---- value: g(x_0) + sum_j <p_j, x_j - x_{j-1}> - delta sum_j c(x_j) |p_j|
    // (the positive equation's; times cost_sign), node terms in T, sums in FP64
    csync<CL>();                                  // every read of red is done (every CTA)
    node_sums(false);
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      if (own[c]) {
        const int k = kbase + tid + c * T_;
        const double w2 = a.cost_sign * a.W2[k];
        const double e0 = (double)x[c][0] - a.c[k];
        acc += 0.5 * w2 * e0 * e0;
        T s = T(0);
#pragma unroll
        for (int j = 1; j <= NM; ++j)
          if (j <= N) s += p[c][j] * (x[c][j] - x[c][j - 1]);
        acc += (double)s;
      }
    }
    csync<CL>();
    if (tid < N && rank == 0) {                   // the node terms, once per point
      const int j = tid + 1;
      T r2 = T(0), n2 = T(0);
      node_total(j, r2, n2);
      acc -= (double)(delta_t * (c0 + c1 * expr<T>(-c2 * r2)) * sqrtr<T>(n2));
    }
    acc = warp_sum<double>(acc);
    if (lane == 0) vred[warp] = acc;
    csync<CL>();
    if (tid == 0 && rank == 0) {
      double v = 0.0;
      for (int w = 0; w < nwarps; ++w) v += vred[w];
      if constexpr (CL > 1)
        for (int w = 0; w < nwarps; ++w) v += peer_vred[w];
      a.V[b] = a.cost_sign * v;
      a.iters[b] = k_it;
      a.status[b] = st;
      count_iterations(a, k_it);
    }
    const T sgn = T(a.cost_sign);
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      if (!own[c]) continue;
      const int k = kbase + tid + c * T_;
#pragma unroll
      for (int j = 0; j <= NM; ++j) {
        if (j <= N) {
          if (a.traj_x != nullptr) a.traj_x[ref.traj + (size_t)j * d + k] = x[c][j];
          if (a.traj_p != nullptr) a.traj_p[ref.traj + (size_t)j * d + k] = (j == 0) ? T(0) : sgn * p[c][j];
        }
      }
    }
  }
  // no CTA of a cluster leaves while the other may still read its shared memory
  if constexpr (CL > 1) csync<CL>();
}

template <typename T, int CPT, int NM, int CL>
hj_status launch_reg(const SolveArgs<T>& a, int threads, cudaStream_t s) {
  // a uniform batch with N = NM takes the instantiation without node guards
  const bool exact = a.Nv == nullptr && a.N == NM;
  auto kern = exact ? lax_eik_reg_kernel<T, CPT, NM, true, CL>
                    : lax_eik_reg_kernel<T, CPT, NM, false, CL>;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HJ_ERR_CUDA;
  if constexpr (CL == 1) {
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, threads, 0) != cudaSuccess)
      return HJ_ERR_CUDA;
    if (bps < 1) return HJ_ERR_UNSUPPORTED;
    int64_t grid = (int64_t)bps * nsm;
    if (a.B < grid) grid = a.B;
    kern<<<(int)grid, threads, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? HJ_OK : HJ_ERR_CUDA;
  } else {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nsm / CL * CL));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;                           // clusters resident at once: the persistent grid
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess) return HJ_ERR_CUDA;
    if (clusters < 1) return HJ_ERR_UNSUPPORTED;
    int64_t nc = clusters;
    if (a.B < nc) nc = a.B;
    cfg.gridDim = dim3((unsigned)(nc * CL));
    if (cudaLaunchKernelEx(&cfg, kern, a) != cudaSuccess) return HJ_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? HJ_OK : HJ_ERR_CUDA;
  }
}

}  // namespace

// Runs the register-resident eikonal kernel when it applies (static bump,
// backward Euler; FP32: d <= 512 with N <= 16, d <= 1024 with N <= 10 and, on a
// cluster of two CTAs, d <= 2048 with N <= 10; FP64: d <= 512 with N <= 10);
// HJ_ERR_UNSUPPORTED otherwise, and the caller takes the shared-memory kernel.
template <typename T>
hj_status launch_eik_reg_solver(const SolveArgs<T>& a, cudaStream_t s) {
  if (a.eik_moving || a.scheme != HJ_SCHEME_BE || a.formulation != HJ_FORM_LAX ||
      a.inner_steps != 1 || a.xb == nullptr)
    return HJ_ERR_UNSUPPORTED;
  if (a.d < 1 || a.N < 1 || a.N > 16) return HJ_ERR_UNSUPPORTED;
  auto threads_for = [](int coords) { return (coords + 31) / 32 * 32; };
  if constexpr (sizeof(T) == 8) {             // FP64 state fits the registers at one coordinate, N <= 10
    if (a.d > kRegMaxThreads || a.N > 10) return HJ_ERR_UNSUPPORTED;
    return launch_reg<T, 1, 10, 1>(a, threads_for(a.d), s);
  } else {
    // two coordinates per thread from d = 64 (half the threads per point, the
    // same work per barrier: d = 100 ran 13.5 against 15.2 ms), one below
    if (a.d >= 64 && a.d <= 2 * kRegMaxThreads && a.N <= 10)
      return launch_reg<T, 2, 10, 1>(a, threads_for((a.d + 1) / 2), s);
    if (a.d <= kRegMaxThreads)
      return a.N <= 10 ? launch_reg<T, 1, 10, 1>(a, threads_for(a.d), s)
                       : launch_reg<T, 1, 16, 1>(a, threads_for(a.d), s);
    if (a.N > 10) return HJ_ERR_UNSUPPORTED;
    if (a.d <= 2 * kRegMaxThreads) return launch_reg<T, 2, 10, 1>(a, threads_for((a.d + 1) / 2), s);
    if (a.d <= 4 * kRegMaxThreads)              // two CTAs, each half of the coordinates
      return launch_reg<T, 2, 10, 2>(a, threads_for(((a.d + 1) / 2 + 1) / 2), s);
    return HJ_ERR_UNSUPPORTED;
  }
}

template hj_status launch_eik_reg_solver<float>(const SolveArgs<float>&, cudaStream_t);
template hj_status launch_eik_reg_solver<double>(const SolveArgs<double>&, cudaStream_t);

}  // namespace hj
