// Coordinate-parallel batched PDHG for the eikonal family at any d (Section 6.1):
// H = c(x)|p|_2, c(x) = c0 + c1 exp(-c2 |x - x_b|^2), Algorithm 1 with the shrink_2
// dual step and one gradient step in x (the scheme the paper runs for its
// eikonal problems, up to d = 2000 in its dimensional-scaling study).
//
// One CTA solves one query point.  Thread t owns the coordinates k = t, t + T,
// ... of every time node, so the difference operator (z_j - z_{j-1} in the dual
// step, p_j - p_{j+1} in the x-step) never leaves the thread.  Only two scalars
// per node involve every coordinate: |x_j - x_b|^2 (for c(x_j)) and |v_j|^2
// (for the shrink of v_j = p_j + sigma (z_j - z_{j-1})).  After the shrink,
// |p_j| = max(|v_j| - lam c(x_j), 0), so the x-step needs no second reduction.
// Per iteration:
//   1. each thread sums its coordinates' parts of both scalars for every node,
//      warps reduce them by shuffles and park them in shared memory;  barrier;
//   2. thread (j - 1) mod T adds the warps' parts for node j and forms that
//      node's shrink factor and x-step coefficient tau delta |p_j| (-2 c1 c2 e_j);
//      barrier;
//   3. each thread, for each of its coordinates: the dual step of every node
//      (old z), then the x-steps of nodes 1..N-1 and the g-prox of x_0, the
//      relaxation, and (test iterations) the squared increments.
// The state x, p, z ([N+1][d], coordinates contiguous, so a warp's accesses are
// consecutive) lives in shared memory when it fits, else in a per-CTA slice of
// a stream-ordered workspace (the d = 2000 problems: L2-resident).
// The negative equation (cost_sign = -1) runs the positive one with -g and
// returns -V and -p, as in Section 6.1.
//
// MIX = true runs the forward-Euler and trapezoid schemes (HJ_SCHEME_FE/TRAP):
// H on interval j is (wR c(x_j) + wL c(x_{j-1}))|p_j|, so node 0's distance to the
// bump is summed too, the shrink threshold takes the averaged speed, the
// x-gradient of node j is grad c(x_j) (wR |p_j| + wL |p_{j+1}|), and x_0 takes the
// gradient step tau delta wL |p_1| grad c(x_0) before the prox of g (two more
// barriers per iteration for the node scalars).
#include <cuda_runtime.h>

#include "hj_internal.cuh"

namespace hj {

namespace {

template <typename T>
__device__ __forceinline__ T expk(T y) { return exp(y); }
template <>
__device__ __forceinline__ float expk<float>(float y) { return __expf(y); }

template <typename T>
__device__ __forceinline__ T sqrtk(T y) { return sqrt(y); }
template <>
__device__ __forceinline__ float sqrtk<float>(float y) { return sqrtf(y); }

// shared memory past the state: red[nwarps][2 (Nmax + 1)] partial sums,
// keep[Nmax + 1], coef[Nmax + 1] node scalars (and, for the mixed schemes,
// the speed c, the gradient factor and |p| of every node: 3 (Nmax + 1)),
// xbs[d], goff[d], ginv[d], then room for 2 nwarps doubles at the next 8-byte
// boundary (tred: the warps' stopping sums, held in the iterate type)
struct EikLayout {
  size_t state;       // elements of one state array: (Nmax + 1) d
  size_t scal;        // elements past the state arrays
  __host__ __device__ EikLayout(int d, int Nmax, int nwarps) {
    state = (size_t)(Nmax + 1) * d;
    scal = (size_t)nwarps * 2 * (Nmax + 1) + 5 * (size_t)(Nmax + 1) + 3 * (size_t)d +
           4 * (size_t)nwarps + 2;                  // 2 nwarps doubles and alignment
  }
};

template <typename T, int NMAX, bool MIX>
__global__ void __launch_bounds__(512) lax_eik_kernel(const SolveArgs<T> a, T* work,
                                                      int state_in_smem) {
  static_assert(!(MIX && NMAX > 0), "the mixed schemes run the generic pass structure");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int d = a.d;
  const int T_ = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = T_ >> 5;
  const EikLayout L(d, a.N, nwarps);
  T* sbase = reinterpret_cast<T*>(smem_raw);
  T* X = state_in_smem ? sbase : work + (size_t)blockIdx.x * 3 * L.state;
  T* P = X + L.state;
  T* Z = P + L.state;
  // red starts 8-byte aligned: the value's FP64 reduction reuses it
  T* red = state_in_smem ? sbase + ((3 * L.state + 1) & ~size_t(1)) : sbase;
  T* keep = red + (size_t)nwarps * 2 * (a.N + 1);
  T* coef = keep + (a.N + 1);
  T* cvv = coef + (a.N + 1);                      // MIX: c(x_j), -2 c1 c2 e_j, |p_j|
  T* evv = cvv + (a.N + 1);
  T* nnv = evv + (a.N + 1);
  T* xbs = nnv + (a.N + 1);
  T* goff = xbs + d;
  T* ginv = goff + d;
  // (an offset from the shared base, so the compiler keeps shared-memory addressing)
  double* tred = reinterpret_cast<double*>(
      smem_raw + ((((size_t)(ginv + d - sbase)) * sizeof(T) + 7) & ~size_t(7)));
  __shared__ unsigned long long s_point;

  for (int k = tid; k < d; k += T_) {
    // cost_sign = -1: the positive equation with the concave initial data -g
    const double w2 = a.cost_sign * a.W2[k], cc = a.c[k];
    xbs[k] = a.xb[k];
    goff[k] = T(a.tau * w2 * cc);
    ginv[k] = T(1.0 / (1.0 + a.tau * w2));
  }
  const T sig = a.sigma_t, tau = a.tau_t, th = a.theta_t;
  const T c0 = a.eik_t[0], c1 = a.eik_t[1], c2 = a.eik_t[2];
  const T wr = a.mix_wr_t, wl = a.mix_wl_t;
  __syncthreads();

  for (;;) {
    __syncthreads();
    if (tid == 0) s_point = draw_item(a);
    __syncthreads();
    const int64_t item = (int64_t)s_point;
    if (item >= a.B) break;
    const PointRef<T> ref = point_ref(a, item);
    const int64_t b = ref.id;
    const int N = ref.N;
    if (N < 1 || N > a.N) {                      // the host never routes such a point here
      if (tid == 0) { a.status[b] = HJ_POINT_INVALID; a.iters[b] = 0; a.V[b] = 0.0; }
      continue;
    }
    const T delta_t = T(a.t[b]) / T(N);
    const T lam = sig * delta_t, taud = tau * delta_t;
    const uint64_t pt = (uint64_t)(a.point_offset + b);

    // ---- initial iterate (Section 6 random guess, or a warm start)
    {
      const InitGuess<T> ig(a.radius);
      for (int k = tid; k < d; k += T_) {
        const double xq = ref.xq[k];
        for (int j = 0; j <= N; ++j) {
          T xv, pv = T(0);
          if (a.warm_x == nullptr) {
            xv = (j < N) ? ig.x(xq, a.seed, pt, j, k) : T(xq);
            if (j >= 1) pv = ig.p(a.seed, pt, j, k);
          } else {
            xv = (j < N) ? a.warm_x[ref.traj + (size_t)j * d + k] : T(xq);
            if (j >= 1) pv = T(a.cost_sign) * a.warm_p[ref.traj + (size_t)j * d + k];
          }
          X[(size_t)j * d + k] = xv;
          P[(size_t)j * d + k] = pv;
          Z[(size_t)j * d + k] = xv;
        }
      }
    }

    // node scalars: |x_j - x_b|^2 and |p_j + sigma (z_j - z_{j-1})|^2 (dual) or
    // |p_j|^2 (value), reduced over the CTA into red
    auto node_sums = [&](bool dual) {
      for (int j = MIX ? 0 : 1; j <= N; ++j) {        // MIX: node 0's distance too
        T pr = T(0), pv = T(0);
        for (int k = tid; k < d; k += T_) {
          const size_t e = (size_t)j * d + k;
          const T y = X[e] - xbs[k];
          pr += y * y;
          if (j > 0) {
            const T v = dual ? P[e] + sig * (Z[e] - Z[e - d]) : P[e];
            pv += v * v;
          }
        }
        pr = warp_sum<T>(pr);
        pv = warp_sum<T>(pv);
        if (lane == 0) {
          red[(size_t)warp * 2 * (N + 1) + 2 * j] = pr;
          red[(size_t)warp * 2 * (N + 1) + 2 * j + 1] = pv;
        }
      }
    };

    int k_it = 0;
    int8_t st = HJ_POINT_MAX_ITER;
    if constexpr (NMAX > 0) node_sums(true);    // the first iteration's node sums
    while (k_it < a.max_iter) {
      ++k_it;
      const bool chk = (k_it % a.check_every == 0) || (k_it == a.max_iter);
      if constexpr (NMAX == 0) node_sums(true);
      __syncthreads();
      if constexpr (MIX) {
        for (int j = tid; j <= N; j += T_) {      // speed and gradient factor of every node
          T r2 = T(0);
          for (int w = 0; w < nwarps; ++w) r2 += red[(size_t)w * 2 * (N + 1) + 2 * j];
          const T e = expk<T>(-c2 * r2);
          cvv[j] = c0 + c1 * e;
          evv[j] = T(-2) * c1 * c2 * e;
        }
        __syncthreads();
        for (int j = 1 + tid; j <= N; j += T_) {  // shrink with the averaged speed
          T n2 = T(0);
          for (int w = 0; w < nwarps; ++w) n2 += red[(size_t)w * 2 * (N + 1) + 2 * j + 1];
          const T n = sqrtk<T>(n2), thr = lam * (wr * cvv[j] + wl * cvv[j - 1]);
          keep[j] = (n > thr) ? (n - thr) / n : T(0);
          nnv[j] = (n > thr) ? n - thr : T(0);
        }
        __syncthreads();
        for (int j = tid; j < N; j += T_) {       // grad c(x_j) (wR |p_j| + wL |p_{j+1}|)
          const T pw = (j == 0) ? wl * nnv[1] : wr * nnv[j] + wl * nnv[j + 1];
          coef[j] = taud * pw * evv[j];
        }
      } else {
        for (int j = 1 + tid; j <= N; j += T_) {
          T r2 = T(0), n2 = T(0);
          for (int w = 0; w < nwarps; ++w) {
            r2 += red[(size_t)w * 2 * (N + 1) + 2 * j];
            n2 += red[(size_t)w * 2 * (N + 1) + 2 * j + 1];
          }
          const T e = expk<T>(-c2 * r2);
          const T n = sqrtk<T>(n2), thr = lam * (c0 + c1 * e);
          keep[j] = (n > thr) ? (n - thr) / n : T(0);
          coef[j] = taud * ((n > thr) ? n - thr : T(0)) * (T(-2) * c1 * c2 * e);
        }
      }
      __syncthreads();
      T rx = T(0), rp = T(0);
      // NMAX > 0: the next iteration's node sums, formed in this pass from the
      // new iterates (node j of every coordinate this thread owns)
      T nr[NMAX > 0 ? NMAX + 1 : 1], nv[NMAX > 0 ? NMAX + 1 : 1];
      if constexpr (NMAX > 0) {
#pragma unroll
        for (int j = 0; j <= NMAX; ++j) { nr[j] = T(0); nv[j] = T(0); }
      }
      for (int k = tid; k < d; k += T_) {
        // dual step of every node with the old z
        T zprev = Z[k];
        for (int j = 1; j <= N; ++j) {
          const size_t e = (size_t)j * d + k;
          const T zj = Z[e];
          const T pn = keep[j] * (P[e] + sig * (zj - zprev));
          if (chk) { const T df = pn - P[e]; rp += df * df; }
          P[e] = pn;
          zprev = zj;
        }
        // primal steps: x_0 (prox of tau g), x_j (j = 1..N-1), relaxation
        const T xb = xbs[k];
        T znew;
        {
          const T xo = X[k];
          const T v0 = MIX ? xo + tau * P[d + k] + coef[0] * (xo - xb) : xo + tau * P[d + k];
          const T xn = (v0 + goff[k]) * ginv[k];
          if (chk) { const T df = xn - xo; rx += df * df; }
          znew = xn + th * (xn - xo);
          Z[k] = znew;
          X[k] = xn;
        }
        if constexpr (NMAX > 0) {
#pragma unroll
          for (int j = 1; j < NMAX; ++j) {
            if (j < N) {
              const size_t e = (size_t)j * d + k;
              const T xo = X[e];
              const T xn = xo - tau * (P[e] - P[e + d]) + coef[j] * (xo - xb);
              if (chk) { const T df = xn - xo; rx += df * df; }
              const T zn = xn + th * (xn - xo);
              Z[e] = zn;
              X[e] = xn;
              const T y = xn - xb, v = P[e] + sig * (zn - znew);
              nr[j] += y * y;
              nv[j] += v * v;
              znew = zn;
            }
          }
          // node N: x_N = z_N = x pinned
          const size_t eN = (size_t)N * d + k;
          const T xN = X[eN], y = xN - xb, v = P[eN] + sig * (xN - znew);
#pragma unroll
          for (int j = 1; j <= NMAX; ++j)
            if (j == N) { nr[j] += y * y; nv[j] += v * v; }
        } else {
          for (int j = 1; j < N; ++j) {
            const size_t e = (size_t)j * d + k;
            const T xo = X[e];
            const T xn = xo - tau * (P[e] - P[e + d]) + coef[j] * (xo - xb);
            if (chk) { const T df = xn - xo; rx += df * df; }
            Z[e] = xn + th * (xn - xo);
            X[e] = xn;
          }
        }
      }
      if constexpr (NMAX > 0) {
        // park the next iteration's node sums (read after the next loop-top barrier;
        // every read of this iteration's sums happened before this pass)
#pragma unroll
        for (int j = 1; j <= NMAX; ++j) {
          if (j <= N) {
            const T pr = warp_sum<T>(nr[j]), pv = warp_sum<T>(nv[j]);
            if (lane == 0) {
              red[(size_t)warp * 2 * (N + 1) + 2 * j] = pr;
              red[(size_t)warp * 2 * (N + 1) + 2 * j + 1] = pv;
            }
          }
        }
      }
      if (chk) {
        // each thread's partial (iterate type) reduced over its warp in that type;
        // the CTA's warp sums accumulated as double-floats (FP32 iterates: as
        // accurate as FP64, on the FP32 pipe) or in FP64, and compared with tol
        T* tsum = reinterpret_cast<T*>(tred);
        const T wx = warp_sum<T>(rx), wp = warp_sum<T>(rp);
        if (lane == 0) { tsum[2 * warp] = wx; tsum[2 * warp + 1] = wp; }
        __syncthreads();
        const int verdict = stop_verdict<T>(a, tsum, nwarps, lane);   // 1 converged, 2 non-finite
        if (verdict == 2) { st = HJ_POINT_NONFINITE; break; }
        if (verdict == 1) { st = HJ_POINT_CONVERGED; break; }
      }
    }

    // ---- value: g(x_0) + sum_j <p_j, x_j - x_{j-1}> - delta sum_j c(x_j) |p_j|
    // (the positive equation's; times cost_sign), node terms in T, sums in FP64
    __syncthreads();
    node_sums(false);
    double acc = 0.0;
    for (int k = tid; k < d; k += T_) {
      const double w2 = a.cost_sign * a.W2[k];
      const double e0 = (double)X[k] - a.c[k];
      acc += 0.5 * w2 * e0 * e0;
      T s = T(0);
      for (int j = 1; j <= N; ++j) {
        const size_t e = (size_t)j * d + k;
        s += P[e] * (X[e] - X[e - d]);
      }
      acc += (double)s;
    }
    __syncthreads();
    for (int j = 1 + tid; j <= N; j += T_) {
      T r2 = T(0), n2 = T(0), rl = T(0);
      for (int w = 0; w < nwarps; ++w) {
        r2 += red[(size_t)w * 2 * (N + 1) + 2 * j];
        n2 += red[(size_t)w * 2 * (N + 1) + 2 * j + 1];
        if (MIX) rl += red[(size_t)w * 2 * (N + 1) + 2 * (j - 1)];
      }
      const T cj = c0 + c1 * expk<T>(-c2 * r2);
      const T cw = MIX ? wr * cj + wl * (c0 + c1 * expk<T>(-c2 * rl)) : cj;
      acc -= (double)(delta_t * cw * sqrtk<T>(n2));
    }
    acc = warp_sum<double>(acc);
    __syncthreads();
    double* vred = reinterpret_cast<double*>(red);   // red is free again (8-byte aligned)
    if (lane == 0) vred[warp] = acc;
    __syncthreads();
    if (tid == 0) {
      double v = 0.0;
      for (int w = 0; w < nwarps; ++w) v += vred[w];
      a.V[b] = a.cost_sign * v;
      a.iters[b] = k_it;
      a.status[b] = st;
      count_iterations(a, k_it);
    }
    if (a.traj_x != nullptr || a.traj_p != nullptr) {
      const T sgn = T(a.cost_sign);
      for (int e = tid; e < (N + 1) * d; e += T_) {
        if (a.traj_x != nullptr) a.traj_x[ref.traj + e] = X[e];
        if (a.traj_p != nullptr) a.traj_p[ref.traj + e] = (e < d) ? T(0) : sgn * P[e];
      }
    }
  }
}

int eik_threads(int d) {
  int t = ((d + 31) / 32) * 32;
  return t < 32 ? 32 : (t > 512 ? 512 : t);
}

template <typename T>
size_t smem_with_state(int d, int N) {
  const EikLayout L(d, N, eik_threads(d) / 32);
  return (((3 * L.state + 1) & ~size_t(1)) + L.scal) * sizeof(T) + 16;
}

template <typename T>
size_t smem_without_state(int d, int N) {
  const EikLayout L(d, N, eik_threads(d) / 32);
  return L.scal * sizeof(T) + 16;
}

constexpr size_t kSmemLimit = 227u * 1024u;
constexpr size_t kWorkspaceCap = size_t(4) << 30;   // workspace bound: fewer CTAs above it

}  // namespace

template <typename T>
size_t eik_cta_smem_bytes(int d, int N) {
  if (d < 1 || d > kMaxDEik || N < 1 || N > kMaxN) return 0;
  const size_t s = smem_with_state<T>(d, N);
  return s <= kSmemLimit ? s : 0;
}

template <typename T>
hj_status launch_eik_cta_solver(const SolveArgs<T>& a, cudaStream_t s) {
  if (a.d < 1 || a.d > kMaxDEik || a.N < 1 || a.N > kMaxN) return HJ_ERR_UNSUPPORTED;
  if (a.xb == nullptr || a.inner_steps != 1 || a.formulation != HJ_FORM_LAX)
    return HJ_ERR_UNSUPPORTED;
  // the state in registers when it fits (backward Euler, d <= 1024, N <= 16)
  {
    const hj_status r = launch_eik_reg_solver<T>(a, s);
    if (r != HJ_ERR_UNSUPPORTED) return r;
  }
  int dev = 0, nsm = 0, max_optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HJ_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
          cudaSuccess)
    return HJ_ERR_CUDA;
  const int threads = eik_threads(a.d);
  const size_t with_state = smem_with_state<T>(a.d, a.N);
  const bool in_smem = with_state <= (size_t)max_optin && with_state <= kSmemLimit;
  const size_t smem = in_smem ? with_state : smem_without_state<T>(a.d, a.N);
  // State in shared memory and N <= 16 (the paper's scaling study runs N = 10):
  // the node sums of the next iteration are formed in the update pass, one pass
  // over the state fewer (d = 100 and 1000: 12 % and 11 % faster).  With the state
  // in the workspace the generic kernel keeps two CTAs per SM (62 registers
  // against the fused kernel's 94), which measured faster (898 against 1119 ms
  // at d = 2000).
  // (the mixed schemes run the generic pass structure)
  auto kern = a.scheme != HJ_SCHEME_BE ? lax_eik_kernel<T, 0, true>
              : (in_smem && a.N <= 16) ? lax_eik_kernel<T, 16, false>
                                       : lax_eik_kernel<T, 0, false>;
  if (smem > (size_t)max_optin) return HJ_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return HJ_ERR_CUDA;
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, threads, smem) != cudaSuccess)
    return HJ_ERR_CUDA;
  if (bps < 1) return HJ_ERR_UNSUPPORTED;
  int64_t grid = (int64_t)bps * nsm;
  if (a.B < grid) grid = a.B;
  T* work = nullptr;
  if (!in_smem) {
    const size_t per_cta = 3 * (size_t)(a.N + 1) * a.d * sizeof(T);
    const int64_t cap = (int64_t)(kWorkspaceCap / per_cta);
    if (cap < 1) return HJ_ERR_UNSUPPORTED;
    if (grid > cap) grid = cap;
    if (cudaMallocAsync(reinterpret_cast<void**>(&work), per_cta * grid, s) != cudaSuccess)
      return HJ_ERR_OOM;
  }
  kern<<<(int)grid, threads, smem, s>>>(a, work, in_smem ? 1 : 0);
  hj_status r = cudaGetLastError() == cudaSuccess ? HJ_OK : HJ_ERR_CUDA;
  if (work != nullptr && cudaFreeAsync(work, s) != cudaSuccess && r == HJ_OK) r = HJ_ERR_CUDA;
  return r;
}

template size_t eik_cta_smem_bytes<float>(int, int);
template size_t eik_cta_smem_bytes<double>(int, int);
template hj_status launch_eik_cta_solver<float>(const SolveArgs<float>&, cudaStream_t);
template hj_status launch_eik_cta_solver<double>(const SolveArgs<double>&, cudaStream_t);

}  // namespace hj
