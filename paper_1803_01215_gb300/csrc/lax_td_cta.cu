// Shared-memory batched PDHG for the tanh-drift Hamiltonian at larger d
// (H = <p, tanh(A x)> + |p|^2/2, Algorithm 1 with the Section 5.3 updates);
// with DRIFT = false the same kernel serves H = |p|^2/2 at any d (the products
// are skipped: a = 0, G = 0).
//
// A CTA holds P points ("slots") at a time; their iterates live in shared
// memory coordinate-major with the slots' node columns side by side
// (X[k][s*Np + j], k = coordinate, j = time node 0..N), so one copy of A serves
// all slots and a thread tile of 4 coordinates x 4 columns reads 16-byte
// vectors.  Per iteration (every active slot advances one iteration):
//   phase A  Y = A X over all columns (register-tiled SIMT product, A^T held in
//            shared memory), epilogue: a = tanh(Y), dual prox
//            p_j <- (p_j + sigma (z_j - z_{j-1}) - lam a) / (1 + lam), lam = sigma delta,
//            and the work array W = (1 - a^2) * p_j.
//   phase B  G = A^T W (second product, A held row-major), epilogue: the primal
//            gradient step x_j <- x_j - tau (p_j - p_{j+1}) + tau delta G_j, the
//            over-relaxation z_j, and the g-prox of x_0.
//   test     per-slot squared increments (warp partials in the iterate type,
//            summed over warps in FP64); a slot tests after every
//            check_every-th of its own iterations.  A finished slot writes its
//            value and trajectory and takes the next point from the work
//            counter while the other slots keep iterating.
#include <cuda_runtime.h>

#include "hj_internal.cuh"

namespace hj {

namespace {

constexpr int kTI = 4;        // coordinates per thread tile
constexpr int kTJ = 4;        // node columns per thread tile
constexpr int kMaxSlots = 4;
constexpr int kMaxWarps = 16; // 512 threads

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
  int dp, Np, NC;           // padded coordinates, padded nodes per slot, columns
  size_t a_elems;           // one copy of A
  size_t s_elems;           // one state array (all slots)
  __host__ __device__ Layout(int d, int N, int P) {
    dp = round4(d);
    Np = round4(N + 1);
    NC = P * Np;
    a_elems = (size_t)d * dp;
    s_elems = (size_t)dp * NC;
  }
};

// Per-slot bookkeeping in static shared memory.
template <typename T>
struct Slots {
  long long id[kMaxSlots];       // launch item, -1 = inactive
  int N[kMaxSlots], k[kMaxSlots], done[kMaxSlots];
  T lam[kMaxSlots], ilam[kMaxSlots], taud[kMaxSlots];
  double delta[kMaxSlots];
  unsigned long long gid[kMaxSlots];
  int8_t st[kMaxSlots];
  T red[kMaxWarps][kMaxSlots][2];
  double vred[kMaxWarps];
};

// TWO: keep both A^T and A in shared memory (vector loads in both products);
// otherwise only A, and the first product reads it with strided scalar loads.
template <typename T, bool TWO, bool DRIFT, int P>
__global__ void __launch_bounds__(512)
lax_td_cta_kernel(const SolveArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Slots<T> S;
  const int d = a.d;
  const Layout L(d, a.N, P);                              // a.N: the largest N of the launch
  const int dp = L.dp, Np = L.Np, NC = L.NC;
  T* Am = reinterpret_cast<T*>(smem_raw);                 // Am[k*dp + i] = A[k][i]
  T* At = TWO ? Am + L.a_elems : Am;                      // At[k*dp + i] = A[i][k]
  T* X = DRIFT ? (TWO ? At + L.a_elems : Am + L.a_elems) : Am;   // no A without drift
  T* Pm = X + L.s_elems;
  T* Z = Pm + L.s_elems;
  T* Wk = Z + L.s_elems;

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
  const T sig = a.sigma_t, tau = a.tau_t, th = a.theta_t;
  const int tilesI = dp / kTI, tilesJ = NC / kTJ, ntiles = tilesI * tilesJ;
  const int tilesPerSlot = Np / kTJ;

  if (DRIFT) {
    for (int e = tid; e < d * dp; e += nthr) {
      const int k = e / dp, i = e - k * dp;
      Am[e] = (i < d) ? a.A[k * d + i] : T(0);
      if (TWO) At[e] = (i < d) ? a.At[k * d + i] : T(0);
    }
  }

  // Take the next point into slot s (all threads; barriers inside).
  auto fill_slot = [&](int s) {
    __syncthreads();
    if (tid == 0) {
      for (;;) {
        const unsigned long long it = atomicAdd(a.counter, 1ull);
        if ((int64_t)it >= a.B) { S.id[s] = -1; break; }
        const PointRef<T> ref = point_ref(a, (int64_t)it);
        if (ref.N < 1 || ref.N > a.N) {           // the host never routes such a point here
          a.status[ref.id] = HJ_POINT_INVALID; a.iters[ref.id] = 0; a.V[ref.id] = 0.0;
          continue;
        }
        S.id[s] = (long long)it;
        S.N[s] = ref.N;
        S.k[s] = 0;
        S.done[s] = 0;
        S.delta[s] = a.t[ref.id] / ref.N;
        const T delta_t = T(a.t[ref.id]) / T(ref.N);
        S.lam[s] = sig * delta_t;
        S.ilam[s] = T(1) / (T(1) + S.lam[s]);
        S.taud[s] = tau * delta_t;
        S.gid[s] = (unsigned long long)(a.point_offset + ref.id);
        S.st[s] = HJ_POINT_MAX_ITER;
        break;
      }
    }
    __syncthreads();
    if (S.id[s] < 0) return;
    const PointRef<T> ref = point_ref(a, (int64_t)S.id[s]);
    const int N = ref.N;
    const uint64_t pt = S.gid[s];
    for (int e = tid; e < dp * Np; e += nthr) {
      const int k = e / Np, j = e - k * Np;
      const int c = k * NC + s * Np + j;
      T xv = T(0), pv = T(0);
      if (k < d && j <= N) {
        const double xq = ref.xq[k];
        if (a.warm_x == nullptr) {
          xv = (j < N) ? T(xq + a.radius * uniform_pm1(a.seed, pt, 0, j, k)) : T(xq);
          pv = (j >= 1) ? T(a.radius * uniform_pm1(a.seed, pt, 1, j, k)) : T(0);
        } else {
          xv = (j < N) ? a.warm_x[ref.traj + (size_t)j * d + k] : T(xq);
          pv = (j >= 1) ? a.warm_p[ref.traj + (size_t)j * d + k] : T(0);
        }
      }
      X[c] = xv; Pm[c] = pv; Z[c] = xv; Wk[c] = T(0);
    }
    __syncthreads();
  };

  // Value (fval of Algorithm 1, FP64) and outputs of the point in slot s.
  auto finish_slot = [&](int s) {
    const PointRef<T> ref = point_ref(a, (int64_t)S.id[s]);
    const int N = ref.N;
    const double delta = S.delta[s];
    const int base = s * Np;
    double acc = 0.0;
    for (int e = tid; e < d * N; e += nthr) {
      const int j = 1 + e / d, i = e - (j - 1) * d;
      double th_y = 0.0;
      if (DRIFT) {
        const double* Ar = a.A64 + (size_t)i * d;
        double y = 0.0;
        for (int k = 0; k < d; ++k) y += Ar[k] * (double)X[k * NC + base + j];
        th_y = tanh(y);
      }
      const double pv = (double)Pm[i * NC + base + j];
      const double dx = (double)X[i * NC + base + j] - (double)X[i * NC + base + j - 1];
      acc += pv * dx - delta * (pv * th_y + 0.5 * pv * pv);
    }
    if (tid < d) {
      const double e0 = (double)X[tid * NC + base] - a.c[tid];
      acc += 0.5 * a.W2[tid] * e0 * e0;
    }
    acc = warp_sum<double>(acc);
    if (lane == 0) S.vred[warp] = acc;
    __syncthreads();
    if (tid == 0) {
      double v = 0.0;
      for (int w = 0; w < nwarps; ++w) v += S.vred[w];
      a.V[ref.id] = v;
      a.iters[ref.id] = S.k[s];
      a.status[ref.id] = S.st[s];
    }
    if (a.traj_x != nullptr || a.traj_p != nullptr) {
      for (int e = tid; e < (N + 1) * d; e += nthr) {
        const int j = e / d, i = e - j * d;
        if (a.traj_x != nullptr) a.traj_x[ref.traj + e] = X[i * NC + base + j];
        if (a.traj_p != nullptr)
          a.traj_p[ref.traj + e] = (j == 0) ? T(0) : Pm[i * NC + base + j];
      }
    }
  };

  for (int s = 0; s < P; ++s) fill_slot(s);

  for (;;) {
    bool any = false;
#pragma unroll
    for (int s = 0; s < P; ++s) any |= (S.id[s] >= 0);
    if (!any) break;
    T rxs[P], rps[P];
#pragma unroll
    for (int s = 0; s < P; ++s) { rxs[s] = T(0); rps[s] = T(0); }

    // ---- phase A: Y = A X, tanh, dual prox, W = (1 - a^2) p
    for (int tile = tid; tile < ntiles; tile += nthr) {
      const int i0 = (tile % tilesI) * kTI, ct = tile / tilesI;
      const int s = ct / tilesPerSlot, j0 = (ct - s * tilesPerSlot) * kTJ;
      if (S.id[s] < 0) continue;
      const int c0 = s * Np + j0, N = S.N[s];
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
        Vec4<T>::load(X + k * NC + c0, xv);
#pragma unroll
        for (int r = 0; r < kTI; ++r)
#pragma unroll
          for (int c = 0; c < kTJ; ++c) acc[r][c] += av[r] * xv[c];
      }
      const T lam = S.lam[s], ilam = S.ilam[s];
      T rp = T(0);
#pragma unroll
      for (int r = 0; r < kTI; ++r) {
        const int i = i0 + r;
#pragma unroll
        for (int c = 0; c < kTJ; ++c) {
          const int j = j0 + c;
          if (i < d && j >= 1 && j <= N) {
            const int e = i * NC + c0 + c;
            const T av = DRIFT ? tanh_c<T>(acc[r][c]) : T(0);
            const T v = Pm[e] + sig * (Z[e] - Z[e - 1]);
            const T pn = (v - lam * av) * ilam;
            const T df = pn - Pm[e];
            rp += df * df;
            Pm[e] = pn;
            Wk[e] = (T(1) - av * av) * pn;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < P; ++q) if (q == s) rps[q] += rp;
    }
    __syncthreads();
    // ---- phase B: G = A^T W, primal gradient step, relaxation; g-prox of x_0
    for (int tile = tid; tile < ntiles; tile += nthr) {
      const int i0 = (tile % tilesI) * kTI, ct = tile / tilesI;
      const int s = ct / tilesPerSlot, j0 = (ct - s * tilesPerSlot) * kTJ;
      if (S.id[s] < 0) continue;
      const int c0 = s * Np + j0, N = S.N[s];
      T acc[kTI][kTJ];
#pragma unroll
      for (int r = 0; r < kTI; ++r)
#pragma unroll
        for (int c = 0; c < kTJ; ++c) acc[r][c] = T(0);
#pragma unroll 4
      for (int k = 0; k < (DRIFT ? d : 0); ++k) {
        T av[kTI], wv[kTJ];
        Vec4<T>::load(Am + k * dp + i0, av);
        Vec4<T>::load(Wk + k * NC + c0, wv);
#pragma unroll
        for (int r = 0; r < kTI; ++r)
#pragma unroll
          for (int c = 0; c < kTJ; ++c) acc[r][c] += av[r] * wv[c];
      }
      const T taud = S.taud[s];
      T rx = T(0);
#pragma unroll
      for (int r = 0; r < kTI; ++r) {
        const int i = i0 + r;
#pragma unroll
        for (int c = 0; c < kTJ; ++c) {
          const int j = j0 + c;
          if (i < d && j >= 1 && j < N) {
            const int e = i * NC + c0 + c;
            const T xo = X[e];
            const T xn = xo - tau * (Pm[e] - Pm[e + 1]) + taud * acc[r][c];
            const T df = xn - xo;
            rx += df * df;
            Z[e] = xn + th * df;
            X[e] = xn;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < P; ++q) if (q == s) rxs[q] += rx;
    }
    for (int e = tid; e < P * d; e += nthr) {             // x_0 of every active slot
      const int s = e / d, i = e - s * d;
      if (S.id[s] < 0) continue;
      const int c = i * NC + s * Np;
      const T w2 = T(a.W2[i]), cc = T(a.c[i]);
      const T xo = X[c];
      const T xn = (xo + tau * Pm[c + 1] + tau * w2 * cc) / (T(1) + tau * w2);
      const T df = xn - xo;
#pragma unroll
      for (int q = 0; q < P; ++q) if (q == s) rxs[q] += df * df;
      Z[c] = xn + th * df;
      X[c] = xn;
    }
    // ---- per-slot increments: warp partials, then FP64 over the warps
#pragma unroll
    for (int s = 0; s < P; ++s) {
      const T sx = warp_sum<T>(rxs[s]), sp = warp_sum<T>(rps[s]);
      if (lane == 0) { S.red[warp][s][0] = sx; S.red[warp][s][1] = sp; }
    }
    __syncthreads();
    // every thread reaches the same decisions from the same shared values
    int kk[P], fin[P];
    int8_t stt[P];
    bool refill = false;
#pragma unroll
    for (int s = 0; s < P; ++s) {
      fin[s] = 0;
      stt[s] = HJ_POINT_MAX_ITER;
      kk[s] = S.k[s] + 1;
      if (S.id[s] < 0) continue;
      const bool chk = (kk[s] % a.check_every == 0) || (kk[s] == a.max_iter);
      if (chk) {
        double sx = 0.0, sp = 0.0;
        for (int w = 0; w < nwarps; ++w) { sx += (double)S.red[w][s][0]; sp += (double)S.red[w][s][1]; }
        if (!(isfinite(sx) && isfinite(sp))) { fin[s] = 1; stt[s] = HJ_POINT_NONFINITE; }
        else if (sx < a.tol && sp < a.tol) { fin[s] = 1; stt[s] = HJ_POINT_CONVERGED; }
        else if (kk[s] == a.max_iter) { fin[s] = 1; }
      }
      refill |= (fin[s] != 0);
    }
    __syncthreads();                                      // every thread has read S.k
    if (tid == 0) {
#pragma unroll
      for (int s = 0; s < P; ++s) {
        if (S.id[s] < 0) continue;
        S.k[s] = kk[s];
        S.done[s] = fin[s];
        if (fin[s]) S.st[s] = stt[s];
      }
    }
    __syncthreads();
    if (refill) {
#pragma unroll
      for (int s = 0; s < P; ++s) {
        if (S.id[s] >= 0 && S.done[s]) {
          finish_slot(s);
          fill_slot(s);
        }
      }
    }
  }
}

template <typename T, bool TWO>
size_t smem_bytes(int d, int N, bool drift, int P) {
  const Layout L(d, N, P);
  const size_t na = drift ? (TWO ? 2 : 1) : 0;
  return (na * L.a_elems + 4 * L.s_elems) * sizeof(T);
}

template <typename T, bool TWO, bool DRIFT, int P>
hj_status launch(const SolveArgs<T>& a, cudaStream_t s, size_t smem) {
  auto kern = lax_td_cta_kernel<T, TWO, DRIFT, P>;
  int dev = 0, nsm = 0, max_optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HJ_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HJ_ERR_CUDA;
  if (cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
      cudaSuccess)
    return HJ_ERR_CUDA;
  if (smem + sizeof(Slots<T>) > (size_t)max_optin) return HJ_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return HJ_ERR_CUDA;
  const Layout L(a.d, a.N, P);
  const int tiles = (L.dp / kTI) * (L.NC / kTJ);
  int threads = ((tiles + 31) / 32) * 32;
  if (threads < 64) threads = 64;
  if (threads > 512) threads = 512;
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, threads, smem) != cudaSuccess)
    return HJ_ERR_CUDA;
  if (bps < 1) return HJ_ERR_UNSUPPORTED;
  const int64_t cap = (int64_t)bps * nsm;
  const int64_t ctas = (a.B + P - 1) / P;
  const int grid = (int)(ctas < cap ? ctas : cap);
  if (grid <= 0) return HJ_OK;
  kern<<<grid, threads, smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? HJ_OK : HJ_ERR_CUDA;
}

constexpr size_t kSmemCap = 227u * 1024u - 4096u;   // room for the static slot table

// The largest slot count (4, 2, 1) whose shared memory fits and that the batch
// can keep busy, preferring both copies of A.
template <typename T, bool DRIFT>
hj_status launch_any(const SolveArgs<T>& a, cudaStream_t s) {
  if (a.B >= 4 * 152) {
    const size_t s4 = smem_bytes<T, true>(a.d, a.N, DRIFT, 4);
    if (s4 <= kSmemCap) return launch<T, true, DRIFT, 4>(a, s, s4);
  }
  if (a.B >= 2 * 152) {
    const size_t s2 = smem_bytes<T, true>(a.d, a.N, DRIFT, 2);
    if (s2 <= kSmemCap) return launch<T, true, DRIFT, 2>(a, s, s2);
  }
  const size_t two = smem_bytes<T, true>(a.d, a.N, DRIFT, 1);
  if (two <= kSmemCap) return launch<T, true, DRIFT, 1>(a, s, two);
  const size_t one = smem_bytes<T, false>(a.d, a.N, DRIFT, 1);
  if (one <= kSmemCap) return launch<T, false, DRIFT, 1>(a, s, one);
  return HJ_ERR_UNSUPPORTED;
}

}  // namespace

template <typename T>
size_t td_cta_smem_bytes(int d, int N, bool drift) {
  const size_t two = smem_bytes<T, true>(d, N, drift, 1);
  if (two <= kSmemCap) return two;
  const size_t one = smem_bytes<T, false>(d, N, drift, 1);
  return one <= kSmemCap ? one : 0;
}

template <typename T>
hj_status launch_td_cta_solver(const SolveArgs<T>& a, bool drift, cudaStream_t s) {
  if (a.d < 1 || a.d > kMaxD || a.N < 1 || a.N > kMaxN || a.inner_steps != 1)
    return HJ_ERR_UNSUPPORTED;
  return drift ? launch_any<T, true>(a, s) : launch_any<T, false>(a, s);
}

template size_t td_cta_smem_bytes<float>(int, int, bool);
template size_t td_cta_smem_bytes<double>(int, int, bool);
template hj_status launch_td_cta_solver<float>(const SolveArgs<float>&, bool, cudaStream_t);
template hj_status launch_td_cta_solver<double>(const SolveArgs<double>&, bool, cudaStream_t);

}  // namespace hj
