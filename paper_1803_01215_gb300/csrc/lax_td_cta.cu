// Shared-memory batched PDHG for the tanh-drift Hamiltonian at larger d
// (H = <p, tanh(A x)> + |p|^2/2, Algorithm 1 with the Section 5.3 updates);
// with DRIFT = false the same kernel serves H = |p|^2/2 at any d (the products
// are skipped: a = 0, G = 0).
//
// One CTA solves one query point at a time; the iterates live in shared memory
// coordinate-major (X[k][j], k = coordinate, j = time node 0..N), so a thread
// tile of 4 coordinates x 4 nodes reads 16-byte vectors.  Per iteration:
//   phase A  Y = A X over all nodes (register-tiled SIMT product, A^T held in
//            shared memory), epilogue: a = tanh(Y), dual prox
//            p_j <- (p_j + sigma (z_j - z_{j-1}) - lam a) / (1 + lam), lam = sigma delta,
//            and the work array W = (1 - a^2) * p_j.
//   phase B  G = A^T W (second product, A held row-major), epilogue: the primal
//            gradient step x_j <- x_j - tau (p_j - p_{j+1}) + tau delta G_j, the
//            over-relaxation z_j, and the g-prox of x_0.
// The squared increments are reduced on test iterations only (over each warp in
// the iterate type, over the warps as double-floats or in FP64).  CTAs
// draw points from a work counter (persistent grid).
//
// MIX = true runs the forward-Euler and trapezoid schemes (HJ_SCHEME_FE/TRAP),
// H on interval j weighted wR at x_j and wL at x_{j-1}: phase A stores
// a = tanh(A x) for every node 0..N in a fifth state array, the dual step
// takes the averaged drift wR a_j + wL a_{j-1}, and W = (1 - a_j^2)(wR p_j +
// wL p_{j+1}) (node 0: wL (1 - a_0^2) p_1) makes A^T W the weighted x-gradient
// of every node, x_0's included (one gradient step before the prox of g).
#include <cuda_runtime.h>

#include "hj_internal.cuh"

namespace hj {

namespace {

constexpr int kTI = 4;   // coordinates per thread tile
constexpr int kTJ = 4;   // nodes per thread tile

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  __device__ __forceinline__ static void load(const float* p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
};
template <>
struct Vec4<double> {
  __device__ __forceinline__ static void load(const double* p, double (&v)[4]) {
    const double2 q0 = *reinterpret_cast<const double2*>(p);
    const double2 q1 = *reinterpret_cast<const double2*>(p + 2);
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
  }
};

__host__ __device__ inline int round4(int v) { return (v + 3) & ~3; }

template <typename T>
__device__ __forceinline__ T tanh_c(T y) { return tanh(y); }
template <>
__device__ __forceinline__ float tanh_c<float>(float y) { return tanhf(y); }

struct Layout {
  int dp, Np;               // padded coordinate count and node count
  size_t a_elems;           // one copy of A
  size_t s_elems;           // one state array
  __host__ __device__ Layout(int d, int N) {
    dp = round4(d);
    Np = round4(N + 1);
    a_elems = (size_t)d * dp;
    s_elems = (size_t)dp * Np;
  }
};

// TWO: keep both A^T and A in shared memory (vector loads in both products);
// otherwise only A, and the first product reads it with strided scalar loads.
template <typename T, bool TWO, bool DRIFT, bool HOPF, bool MIX>
__global__ void __launch_bounds__(512)
lax_td_cta_kernel(const SolveArgs<T> a) {
  static_assert(!(MIX && (HOPF || !DRIFT)), "the mixed schemes: Lax form, tanh drift");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int d = a.d;
  const Layout L(d, a.N);                                 // a.N: the largest N of the launch
  const int dp = L.dp;
  T* Am = reinterpret_cast<T*>(smem_raw);                 // Am[k*dp + i] = A[k][i]
  T* At = TWO ? Am + L.a_elems : Am;                      // At[k*dp + i] = A[i][k]
  T* X = DRIFT ? (TWO ? At + L.a_elems : Am + L.a_elems) : Am;   // no A without drift
  T* P = X + L.s_elems;
  T* Z = P + L.s_elems;
  T* Wk = Z + L.s_elems;
  T* Asv = Wk + L.s_elems;                                  // MIX: tanh(A x) of every node
  double* red = reinterpret_cast<double*>(Wk + (MIX ? 2 : 1) * L.s_elems);  // [2 * nwarps]
  double* tred = red;                                       // [2 * nwarps] stopping test
  T* hsv = reinterpret_cast<T*>(red + 32);                  // Hopf form: sigma / W^2, sigma c
  T* hcv = hsv + dp;
  __shared__ unsigned long long s_point;

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;

  if (DRIFT) {
    for (int e = tid; e < d * dp; e += nthr) {
      const int k = e / dp, i = e - k * dp;
      Am[e] = (i < d) ? a.A[k * d + i] : T(0);
      if (TWO) At[e] = (i < d) ? a.At[k * d + i] : T(0);
    }
  }

  for (int i = threadIdx.x; i < dp; i += blockDim.x) {
    hsv[i] = (HOPF && i < d) ? T(a.sigma / a.W2[i]) : T(0);
    hcv[i] = (i < d) ? T(a.sigma * a.c[i]) : T(0);
  }
  const T sig = a.sigma_t, tau = a.tau_t, th = a.theta_t;
  const T wr = a.mix_wr_t, wl = a.mix_wl_t;

  for (;;) {
    __syncthreads();
    if (tid == 0) s_point = draw_item(a);
    __syncthreads();
    const int64_t item = (int64_t)s_point;
    if (item >= a.B) break;
    const PointRef<T> ref = point_ref(a, item);
    const int64_t b = ref.id;
    const int N = ref.N;
    if (N < 1 || N > a.N) {                                // the host never routes such a point here
      if (tid == 0) { a.status[b] = HJ_POINT_INVALID; a.iters[b] = 0; a.V[b] = 0.0; }
      continue;
    }
    const int Np = round4(N + 1);
    const int tilesI = dp / kTI, tilesJ = Np / kTJ;
    const int ntiles = tilesI * tilesJ;
    const double delta = a.t[b] / N;                      // value epilogue only
    const T delta_t = T(a.t[b]) / T(N);
    const T lam = sig * delta_t, taud = tau * delta_t;
    const T ilam = T(1) / (T(1) + lam);
    const uint64_t pt = (uint64_t)(a.point_offset + b);

    // ---- initial iterate (Section 6 random guess, or a warm start)
    for (int e = tid; e < dp * Np; e += nthr) {
      const int k = e / Np, j = e - k * Np;
      T xv = T(0), pv = T(0);
      if (k < d && j <= N && !(HOPF && j == 0)) {         // Hopf: x_0 is not a variable (0)
        const double xq = ref.xq[k];
        if (a.warm_x == nullptr) {
          const InitGuess<T> ig(a.radius);
          xv = (j < N) ? ig.x(xq, a.seed, pt, j, k) : T(xq);
          pv = (j >= 1) ? ig.p(a.seed, pt, j, k) : T(0);
        } else {
          xv = (j < N) ? a.warm_x[ref.traj + (size_t)j * d + k] : T(xq);
          pv = (j >= 1) ? a.warm_p[ref.traj + (size_t)j * d + k] : T(0);
        }
      }
      X[e] = xv; P[e] = pv; Z[e] = xv; Wk[e] = T(0);
    }
    __syncthreads();

    int k_it = 0;
    int8_t st = HJ_POINT_MAX_ITER;
    while (k_it < a.max_iter) {
      ++k_it;
      const bool chk = (k_it % a.check_every == 0) || (k_it == a.max_iter);
      T rx = T(0), rp = T(0);
      // ---- phase A: Y = A X, tanh, dual prox, W = (1 - a^2) p
      for (int tile = tid; tile < ntiles; tile += nthr) {
        const int i0 = (tile % tilesI) * kTI, j0 = (tile / tilesI) * kTJ;
        T acc[kTI][kTJ];
#pragma unroll
        for (int r = 0; r < kTI; ++r)
#pragma unroll
          for (int c = 0; c < kTJ; ++c) acc[r][c] = T(0);
#pragma unroll 4
        for (int k = 0; k < (DRIFT ? d : 0); ++k) {
          T av[kTI], xv[kTJ];
          if (TWO) {
            Vec4<T>::load(At + k * dp + i0, av);
          } else {
#pragma unroll
            for (int r = 0; r < kTI; ++r) av[r] = (i0 + r < d) ? Am[(i0 + r) * dp + k] : T(0);
          }
          Vec4<T>::load(X + k * Np + j0, xv);
#pragma unroll
          for (int r = 0; r < kTI; ++r)
#pragma unroll
            for (int c = 0; c < kTJ; ++c) acc[r][c] += av[r] * xv[c];
        }
        if constexpr (MIX) {                      // a of every node; the dual step below
#pragma unroll
          for (int r = 0; r < kTI; ++r)
#pragma unroll
            for (int c = 0; c < kTJ; ++c)
              if (i0 + r < d && j0 + c <= N) Asv[(i0 + r) * Np + j0 + c] = tanh_c<T>(acc[r][c]);
        } else {
#pragma unroll
        for (int r = 0; r < kTI; ++r) {
          const int i = i0 + r;
#pragma unroll
          for (int c = 0; c < kTJ; ++c) {
            const int j = j0 + c;
            if (i < d && j >= 1 && j <= N) {
              const int e = i * Np + j;
              const T av = DRIFT ? tanh_c<T>(acc[r][c]) : T(0);
              const T v = P[e] + sig * (Z[e] - Z[e - 1]);
              const T pn = (HOPF && j == 1)         // Hopf node 1: prox of sigma g* + lam H
                               ? (v - hcv[i] - lam * av) / (T(1) + lam + hsv[i])
                               : (v - lam * av) * ilam;
              if (chk) { const T df = pn - P[e]; rp += df * df; }
              P[e] = pn;
              Wk[e] = (T(1) - av * av) * pn;
            }
          }
        }
        }
      }
      if constexpr (MIX) {
        __syncthreads();
        // dual step with the averaged drift: (1 + lam) p = v - lam (wR a_j + wL a_{j-1})
        for (int e2 = tid; e2 < d * N; e2 += nthr) {
          const int i = e2 / N, j = 1 + (e2 - i * N);
          const int e = i * Np + j;
          const T v = P[e] + sig * (Z[e] - Z[e - 1]);
          const T pn = (v - lam * (wr * Asv[e] + wl * Asv[e - 1])) * ilam;
          if (chk) { const T df = pn - P[e]; rp += df * df; }
          P[e] = pn;
        }
        __syncthreads();
        // W = (1 - a_j^2)(wR p_j + wL p_{j+1}), j = 1..N-1; node 0: wL (1 - a_0^2) p_1
        for (int e2 = tid; e2 < d * N; e2 += nthr) {
          const int i = e2 / N, j = e2 - i * N;
          const int e = i * Np + j;
          const T av = Asv[e];
          const T pw = (j == 0) ? wl * P[e + 1] : wr * P[e] + wl * P[e + 1];
          Wk[e] = (T(1) - av * av) * pw;
        }
      }
      __syncthreads();
      // ---- phase B: G = A^T W, primal gradient step, relaxation; g-prox of x_0
      for (int tile = tid; tile < ntiles; tile += nthr) {
        const int i0 = (tile % tilesI) * kTI, j0 = (tile / tilesI) * kTJ;
        T acc[kTI][kTJ];
#pragma unroll
        for (int r = 0; r < kTI; ++r)
#pragma unroll
          for (int c = 0; c < kTJ; ++c) acc[r][c] = T(0);
#pragma unroll 4
        for (int k = 0; k < (DRIFT ? d : 0); ++k) {
          T av[kTI], wv[kTJ];
          Vec4<T>::load(Am + k * dp + i0, av);
          Vec4<T>::load(Wk + k * Np + j0, wv);
#pragma unroll
          for (int r = 0; r < kTI; ++r)
#pragma unroll
            for (int c = 0; c < kTJ; ++c) acc[r][c] += av[r] * wv[c];
        }
#pragma unroll
        for (int r = 0; r < kTI; ++r) {
          const int i = i0 + r;
#pragma unroll
          for (int c = 0; c < kTJ; ++c) {
            const int j = j0 + c;
            if (i < d && j >= 1 && j < N) {
              const int e = i * Np + j;
              const T xo = X[e];
              const T xn = xo - tau * (P[e] - P[e + 1]) + taud * acc[r][c];
              if (chk) { const T df = xn - xo; rx += df * df; }
              Z[e] = xn + th * (xn - xo);
              X[e] = xn;
            } else if (MIX && i < d && j == 0) {
              // x_0: gradient step on -delta wL H(x_0, p_1) (in W), then the prox of g
              const int e = i * Np;
              const T w2 = T(a.W2[i]), cc = T(a.c[i]);
              const T xo = X[e];
              const T xn = (xo + tau * P[e + 1] + taud * acc[r][c] + tau * w2 * cc) /
                           (T(1) + tau * w2);
              if (chk) { const T df = xn - xo; rx += df * df; }
              Z[e] = xn + th * (xn - xo);
              X[e] = xn;
            }
          }
        }
      }
      if (!HOPF && !MIX && tid < d) {
        const int e = tid * Np;
        const T w2 = T(a.W2[tid]), cc = T(a.c[tid]);
        const T xo = X[e];
        const T xn = (xo + tau * P[e + 1] + tau * w2 * cc) / (T(1) + tau * w2);
        if (chk) { const T df = xn - xo; rx += df * df; }
        Z[e] = xn + th * (xn - xo);
        X[e] = xn;
      }
      // each thread's partial (iterate type) reduced over its warp in that type;
      // the CTA's warp sums accumulated as double-floats (FP32 iterates: as
      // accurate as FP64, on the FP32 pipe) or in FP64, and compared with tol
      T* tsum = reinterpret_cast<T*>(tred);
      if (chk) {
        const T wx = warp_sum<T>(rx), wp = warp_sum<T>(rp);
        if (lane == 0) { tsum[2 * warp] = wx; tsum[2 * warp + 1] = wp; }
      }
      __syncthreads();
      if (chk) {
        const int verdict = stop_verdict<T>(a, tsum, nwarps, lane);   // 1 converged, 2 non-finite
        if (verdict == 2) { st = HJ_POINT_NONFINITE; break; }
        if (verdict == 1) { st = HJ_POINT_CONVERGED; break; }
      }
    }

    // ---- value g(x_0) + sum_j <p_j, x_j - x_{j-1}> - delta sum_j H(x_j, p_j):
    // FP64 iterates evaluate every term in FP64; FP32 iterates form each
    // (coordinate, node) term in FP32 (A x from the FP32 copy of A); the sum is FP64
    double acc = 0.0;
    for (int e = tid; e < d * N; e += nthr) {
      const int j = 1 + e / d, i = e - (j - 1) * d;
      // the drift at x_j, and (MIX) weighted with the one at x_{j-1}
      if constexpr (sizeof(T) == 4) {
        T th_y = T(0);
        if (DRIFT) {
          T y = T(0), yl = T(0);
          for (int k = 0; k < d; ++k) {
            y += Am[i * dp + k] * X[k * Np + j];
            if (MIX) yl += Am[i * dp + k] * X[k * Np + j - 1];
          }
          th_y = MIX ? wr * tanh_c<T>(y) + wl * tanh_c<T>(yl) : tanh_c<T>(y);
        }
        const T pv = P[i * Np + j];
        const T dx = X[i * Np + j] - X[i * Np + j - 1];
        acc += (double)(pv * dx - delta_t * (pv * th_y + T(0.5) * pv * pv));
      } else {
        double th_y = 0.0;
        if (DRIFT) {
          const double* Ar = a.A64 + (size_t)i * d;
          double y = 0.0, yl = 0.0;
          for (int k = 0; k < d; ++k) {
            y += Ar[k] * (double)X[k * Np + j];
            if (MIX) yl += Ar[k] * (double)X[k * Np + j - 1];
          }
          th_y = MIX ? a.mix_wr * tanh(y) + a.mix_wl * tanh(yl) : tanh(y);
        }
        const double pv = (double)P[i * Np + j];
        const double dx = (double)X[i * Np + j] - (double)X[i * Np + j - 1];
        acc += pv * dx - delta * (pv * th_y + 0.5 * pv * pv);
      }
    }
    if (tid < d) {
      if (HOPF) {                                         // -g*(p_1)
        const double p1 = (double)P[tid * Np + 1];
        acc -= p1 * a.c[tid] + 0.5 * p1 * p1 / a.W2[tid];
      } else {
        const double e0 = (double)X[tid * Np] - a.c[tid];
        acc += 0.5 * a.W2[tid] * e0 * e0;
      }
    }
    acc = warp_sum<double>(acc);
    __syncthreads();
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (tid == 0) {
      double v = 0.0;
      for (int w = 0; w < nwarps; ++w) v += red[w];
      a.V[b] = v;
      a.iters[b] = k_it;
      a.status[b] = st;
      count_iterations(a, k_it);
    }
    if (a.traj_x != nullptr || a.traj_p != nullptr) {
      for (int e = tid; e < (N + 1) * d; e += nthr) {
        const int j = e / d, i = e - j * d;
        if (a.traj_x != nullptr)                          // Hopf: x_0 = c + p_1 / W^2
          a.traj_x[ref.traj + e] = (HOPF && j == 0)
                                       ? T(a.c[i] + (double)P[i * Np + 1] / a.W2[i])
                                       : X[i * Np + j];
        if (a.traj_p != nullptr) a.traj_p[ref.traj + e] = (j == 0) ? T(0) : P[i * Np + j];
      }
    }
  }
}

template <typename T, bool TWO>
size_t smem_bytes(int d, int N, bool drift, bool mix = false) {
  const Layout L(d, N);
  const size_t na = drift ? (TWO ? 2 : 1) : 0;
  return (na * L.a_elems + (mix ? 5 : 4) * L.s_elems + 2 * L.dp) * sizeof(T) +
         2 * 16 * sizeof(double);
}

template <typename T, bool TWO, bool DRIFT, bool HOPF, bool MIX>
hj_status launch_form(const SolveArgs<T>& a, cudaStream_t s, size_t smem) {
  auto kern = lax_td_cta_kernel<T, TWO, DRIFT, HOPF, MIX>;
  int dev = 0, nsm = 0, max_optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HJ_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HJ_ERR_CUDA;
  if (cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
      cudaSuccess)
    return HJ_ERR_CUDA;
  if (smem > (size_t)max_optin) return HJ_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return HJ_ERR_CUDA;
  const Layout L(a.d, a.N);
  const int tiles = (L.dp / kTI) * (L.Np / kTJ);
  int threads = ((tiles + 31) / 32) * 32;
  if (threads < 64) threads = 64;
  if (threads > 512) threads = 512;
  if (threads < a.d) threads = ((a.d + 31) / 32) * 32;   // x_0 update: one thread per coordinate
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, threads, smem) != cudaSuccess)
    return HJ_ERR_CUDA;
  if (bps < 1) return HJ_ERR_UNSUPPORTED;
  const int64_t cap = (int64_t)bps * nsm;
  const int grid = (int)(a.B < cap ? a.B : cap);
  kern<<<grid, threads, smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? HJ_OK : HJ_ERR_CUDA;
}

template <typename T, bool TWO, bool DRIFT>
hj_status launch(const SolveArgs<T>& a, cudaStream_t s, size_t smem) {
  if constexpr (DRIFT) {
    if (a.scheme != HJ_SCHEME_BE) {
      if (a.formulation == HJ_FORM_HOPF) return HJ_ERR_UNSUPPORTED;
      return launch_form<T, TWO, DRIFT, false, true>(a, s, smem);
    }
  }
  return a.formulation == HJ_FORM_HOPF ? launch_form<T, TWO, DRIFT, true, false>(a, s, smem)
                                       : launch_form<T, TWO, DRIFT, false, false>(a, s, smem);
}

}  // namespace

template <typename T>
size_t td_cta_smem_bytes(int d, int N, bool drift, bool mix) {
  mix = mix && drift;
  const size_t two = smem_bytes<T, true>(d, N, drift, mix);
  if (two <= 227u * 1024u) return two;
  const size_t one = smem_bytes<T, false>(d, N, drift, mix);
  return one <= 227u * 1024u ? one : 0;
}

template <typename T>
hj_status launch_td_cta_solver(const SolveArgs<T>& a, bool drift, cudaStream_t s) {
  if (a.d < 1 || a.d > kMaxD || a.N < 1 || a.N > kMaxN || a.inner_steps != 1)
    return HJ_ERR_UNSUPPORTED;
  const bool mix = drift && a.scheme != HJ_SCHEME_BE;   // the tiled kernel: backward Euler
  if constexpr (sizeof(T) == 4) {
    if (drift && !mix) {
      const hj_status r = launch_td_tile_solver(a, s);
      if (r != HJ_ERR_UNSUPPORTED) return r;
    }
  }
  if (!drift) {
    const size_t sm = smem_bytes<T, false>(a.d, a.N, false);
    return sm <= 227u * 1024u ? launch<T, false, false>(a, s, sm) : HJ_ERR_UNSUPPORTED;
  }
  const size_t two = smem_bytes<T, true>(a.d, a.N, true, mix);
  if (two <= 227u * 1024u) return launch<T, true, true>(a, s, two);
  const size_t one = smem_bytes<T, false>(a.d, a.N, true, mix);
  if (one <= 227u * 1024u) return launch<T, false, true>(a, s, one);
  return HJ_ERR_UNSUPPORTED;
}

template size_t td_cta_smem_bytes<float>(int, int, bool, bool);
template size_t td_cta_smem_bytes<double>(int, int, bool, bool);
template hj_status launch_td_cta_solver<float>(const SolveArgs<float>&, bool, cudaStream_t);
template hj_status launch_td_cta_solver<double>(const SolveArgs<double>&, bool, cudaStream_t);

}  // namespace hj
