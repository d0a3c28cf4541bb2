// Register-tiled batched PDHG for the tanh-drift Hamiltonian with FP32 iterates:
// H = <p, tanh(A x)> + |p|^2/2 (Algorithm 1 with the Section 5.3 updates).
//
// A group of G warps solves one query point.  Each thread owns a fixed tile of
// 4 coordinates x TJ time nodes (TJ = 4 for d <= 64: 128 registers, twice the
// warps per SM, groups of up to 16 warps; TJ = 8 above, where the larger groups
// measured slower) and keeps that tile's x, p and z in registers
// for the whole solve (thread t of the group: within each block of 4*TIc
// threads, i-tile = u / 4 and j-tile = 4 * block + u % 4, so a quarter-warp
// covers 2 i-tiles x 4 j-tiles and its 16-byte operand loads stay cheap).  Only
// what other threads need goes through shared memory:
//   Xs[k][j-1]   the x iterate of nodes 1..N (operand of A x), published after
//                the primal step;
//   Ws[k][j-1]   W = (1 - a^2) p (operand of A^T W), published after the dual step;
//   Zb, Pb       the z of each tile's last node and the p of its first node,
//                the neighbour terms z_{j-1} and p_{j+1} across tile boundaries.
// Per iteration:
//   phase A  Y = A X over the tile (k-loop over 16-byte loads of A^T and Xs),
//            then a = tanh(Y), the dual prox
//            p_j <- (p_j + sigma (z_j - z_{j-1}) - lam a) / (1 + lam), lam = sigma delta,
//            and W = (1 - a^2) p_j;
//   phase B  G = A^T W, then x_j <- x_j - tau (p_j - p_{j+1}) + tau delta G_j,
//            z_j = x_j + theta (x_j - x_j_old), and the g-prox of x_0 (held by
//            the threads of the first node tile).
// x_N stays pinned at the query point.  One group barrier after each phase
// (__syncwarp when G = 1).  On test iterations each thread's squared
// increments (its tile, FP32) are reduced over the warp in FP32, and the
// group's warp sums are accumulated as double-floats (error-free TwoSum: as
// accurate as FP64) and compared with tol; the value's (coordinate, node) terms
// are FP32 and their sum FP64.  Groups take points from the work
// counter (persistent grid); the CTA's groups share one copy of A and A^T.
#include <cuda_runtime.h>

#include "hj_internal.cuh"

namespace hj {

namespace {

constexpr int kTI = 4;   // coordinates per tile

template <int TJ>
struct TileLayout {
  int d, dp, TIc, TJc, Ns;
  size_t head_bytes;     // per-group item slots, g-prox and Hopf node-1 constants
  size_t a_floats;       // A^T and A
  size_t grp_floats;     // Xs, Ws, Zb, Pb, reductions of one group
  __host__ __device__ TileLayout(int d_, int Nmax, int G, int M) {
    d = d_;
    dp = (d + 3) & ~3;
    TIc = dp / kTI;
    TJc = (Nmax + TJ - 1) / TJ;
    Ns = TJ * TJc + 4;                               // row stride of Xs and Ws
    head_bytes = (size_t)((M * 8 + 15) / 16) * 16 + 4 * (size_t)dp * sizeof(float);
    a_floats = 2 * (size_t)d * dp;
    grp_floats = 2 * (size_t)dp * Ns + 2 * (size_t)TJc * dp + 6 * (size_t)G;   // + 3G doubles
    grp_floats = (grp_floats + 3) & ~size_t(3);       // keep 16-byte alignment
  }
  __host__ __device__ size_t bytes(int M) const {
    return head_bytes + (a_floats + (size_t)M * grp_floats) * sizeof(float);
  }
};

// threads a point needs: tiles laid out in blocks of 4 j-tiles
__host__ __device__ inline int tile_slots(int d, int Nmax, int TJ) {
  const int TIc = ((d + 3) & ~3) / kTI, TJc = (Nmax + TJ - 1) / TJ;
  return 4 * TIc * ((TJc + 3) / 4);
}

template <int G>
__device__ __forceinline__ void group_barrier(int grp) {
  if constexpr (G == 1) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(32 * G) : "memory");
  }
}

template <int TJ>
__device__ __forceinline__ void loadv(const float* p, float (&v)[TJ]) {
#pragma unroll
  for (int q = 0; q < TJ / 4; ++q) {
    const float4 a = *reinterpret_cast<const float4*>(p + 4 * q);
    v[4 * q] = a.x; v[4 * q + 1] = a.y; v[4 * q + 2] = a.z; v[4 * q + 3] = a.w;
  }
}
template <int TJ>
__device__ __forceinline__ void storev(float* p, const float (&v)[TJ]) {
#pragma unroll
  for (int q = 0; q < TJ / 4; ++q)
    *reinterpret_cast<float4*>(p + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// acc[r][c] = sum_k M[k][i0 + r] * S[k][c0 + c], k < d (M k-major with stride dp).
// The accumulators are updated in pairs of nodes by the packed FP32 fma
// (__ffma2_rn: each lane rounded once, bitwise the same as two fmaf), half the
// issue slots of scalar fmaf.
template <int TJ>
__device__ __forceinline__ void tile_product(const float* M, const float* S, int d, int dp,
                                             int Ns, int i0, int c0,
                                             float (&acc)[kTI][TJ]) {
  float2 acc2[kTI][TJ / 2];
#pragma unroll
  for (int r = 0; r < kTI; ++r)
#pragma unroll
    for (int q = 0; q < TJ / 2; ++q) acc2[r][q] = make_float2(0.f, 0.f);
  const float* mp = M + i0;
  const float* sp = S + c0;
  // k-steps unrolled 4 (four-node tiles, at 128 registers) or 8 (eight-node
  // tiles: d = 100 ran 290.7 against 297.7 ms; four-node tiles lost at 8)
#pragma unroll(TJ == 4 ? 4 : 8)
  for (int k = 0; k < d; ++k) {
    const float4 a = *reinterpret_cast<const float4*>(mp);
    float2 s2[TJ / 2];
#pragma unroll
    for (int q = 0; q < TJ / 4; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(sp + 4 * q);
      s2[2 * q] = make_float2(v.x, v.y);
      s2[2 * q + 1] = make_float2(v.z, v.w);
    }
    mp += dp;
    sp += Ns;
    const float av[kTI] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int r = 0; r < kTI; ++r) {
      const float2 ar = make_float2(av[r], av[r]);
#pragma unroll
      for (int q = 0; q < TJ / 2; ++q) acc2[r][q] = __ffma2_rn(ar, s2[q], acc2[r][q]);
    }
  }
#pragma unroll
  for (int r = 0; r < kTI; ++r)
#pragma unroll
    for (int q = 0; q < TJ / 2; ++q) { acc[r][2 * q] = acc2[r][q].x; acc[r][2 * q + 1] = acc2[r][q].y; }
}

// Four-node tiles are held to 128 registers: CTAs of max(128, 32 G) threads,
// 65536 / (128 x threads) of them per SM (16 warps).  Eight-node tiles: up to
// 256 threads, about 240 registers.
template <int TJ, int G>
constexpr int tile_cta_threads() { return TJ == 4 ? (32 * G > 128 ? 32 * G : 128) : 256; }
template <int TJ, int G>
constexpr int tile_min_ctas() { return TJ == 4 ? 65536 / (128 * tile_cta_threads<TJ, G>()) : 1; }

template <int TJ, int G, bool TH1, bool HOPF>
__global__ void __launch_bounds__(tile_cta_threads<TJ, G>(), tile_min_ctas<TJ, G>())
lax_td_tile_kernel(const SolveArgs<float> a, int M) {
  constexpr int kTJ = TJ;
  extern __shared__ __align__(16) unsigned char smem[];
  const TileLayout<TJ> L(a.d, a.N, G, M);
  const int d = L.d, dp = L.dp, Ns = L.Ns;
  unsigned long long* items = reinterpret_cast<unsigned long long*>(smem);
  float* goff = reinterpret_cast<float*>(smem + (size_t)((M * 8 + 15) / 16) * 16);
  float* ginv = goff + dp;
  float* hs = ginv + dp;                          // Hopf form: sigma / W^2 and sigma c
  float* hc = hs + dp;
  float* At = hc + dp;                            // At[k*dp + i] = A[i][k]
  float* Am = At + (size_t)d * dp;                // Am[k*dp + i] = A[k][i]
  const int grp = (int)threadIdx.x / (32 * G);
  float* Xs = Am + (size_t)d * dp + (size_t)grp * L.grp_floats;
  float* Ws = Xs + (size_t)dp * Ns;
  float* Zb = Ws + (size_t)dp * Ns;               // Zb[jt*dp + i]
  float* Pb = Zb + (size_t)L.TJc * dp;            // Pb[jt*dp + i]
  // [2G] floats (test sums, in the space of 2G doubles) then [G] doubles (value);
  // Pb + TJc dp floats keeps 16-byte alignment
  float* tred = Pb + (size_t)L.TJc * dp;
  double* vred = reinterpret_cast<double*>(tred) + 2 * G;

  for (int e = threadIdx.x; e < d * dp; e += blockDim.x) {
    const int k = e / dp, i = e - k * dp;
    At[e] = (i < d) ? a.At[k * d + i] : 0.f;
    Am[e] = (i < d) ? a.A[k * d + i] : 0.f;
  }
  for (int i = threadIdx.x; i < dp; i += blockDim.x) {
    const double w2 = i < d ? a.W2[i] : 0.0, cc = i < d ? a.c[i] : 0.0;
    goff[i] = (float)(a.tau * w2 * cc);
    ginv[i] = (float)(1.0 / (1.0 + a.tau * w2));
    hs[i] = (HOPF && i < d) ? (float)(a.sigma / w2) : 0.f;
    hc[i] = (float)(a.sigma * cc);
  }
  __syncthreads();
  if (grp >= M) return;                           // no thread of a partial group exists

  const int t = (int)threadIdx.x - grp * 32 * G;  // thread within the group
  const int lane = t & 31, wig = t >> 5;
  const int blk = 4 * L.TIc;
  const int u = t % blk, jg = t / blk;
  const int it = u >> 2, jt = 4 * jg + (u & 3);
  const bool tile_ok = it < L.TIc && jt < L.TJc;
  const int i0 = it * kTI, c0 = jt * kTJ, j0 = 1 + c0;   // nodes j0..j0+TJ-1 <-> Xs columns c0..c0+TJ-1
  const float sig = a.sigma_t, tau = a.tau_t, th = a.theta_t;

  for (;;) {
    group_barrier<G>(grp);
    if (t == 0) items[grp] = draw_item(a);
    group_barrier<G>(grp);
    const int64_t item = (int64_t)items[grp];
    if (item >= a.B) break;
    const PointRef<float> ref = point_ref(a, item);
    const int64_t b = ref.id;
    const int N = ref.N;
    if (N < 1 || N > a.N) {                      // the host never routes such a point here
      if (t == 0) { a.status[b] = HJ_POINT_INVALID; a.iters[b] = 0; a.V[b] = 0.0; }
      continue;
    }
    const bool act = tile_ok && c0 < N;           // the tile holds nodes of this point
    const float delta_t = (float)a.t[b] / (float)N;
    const float lam = sig * delta_t, taud = tau * delta_t;
    const float ilam = 1.f / (1.f + lam);
    const uint64_t pt = (uint64_t)(a.point_offset + b);

    float x[kTI][kTJ], p[kTI][kTJ], z[kTI][kTJ], x0[kTI], z0[kTI];
    {
      const InitGuess<float> ig(a.radius);
#pragma unroll
      for (int r = 0; r < kTI; ++r) {
        const int i = i0 + r;
        const bool row = act && i < d;
        const double xq = row ? ref.xq[i] : 0.0;
#pragma unroll
        for (int c = 0; c < kTJ; ++c) {
          const int j = j0 + c;
          float xv = 0.f, pv = 0.f;
          if (row && j <= N) {
            if (a.warm_x == nullptr) {
              xv = (j < N) ? ig.x(xq, a.seed, pt, j, i) : (float)xq;
              pv = ig.p(a.seed, pt, j, i);
            } else {
              xv = (j < N) ? a.warm_x[ref.traj + (size_t)j * d + i] : (float)xq;
              pv = a.warm_p[ref.traj + (size_t)j * d + i];
            }
          }
          x[r][c] = xv; p[r][c] = pv; z[r][c] = xv;
        }
        float x0v = 0.f;                          // Hopf: x_0 is not a variable (0)
        if (row && jt == 0 && !HOPF)
          x0v = (a.warm_x == nullptr) ? ig.x(xq, a.seed, pt, 0, i) : a.warm_x[ref.traj + i];
        x0[r] = x0v; z0[r] = x0v;
      }
    }
    if (act) {
#pragma unroll
      for (int r = 0; r < kTI; ++r) {
        storev<kTJ>(Xs + (size_t)(i0 + r) * Ns + c0, x[r]);
        Zb[jt * dp + i0 + r] = z[r][kTJ - 1];
      }
    }
    group_barrier<G>(grp);

    // one iteration; CHK adds the squared increments (test iterations only)
    auto step = [&](auto chk_tag, float& rx, float& rp) {
      constexpr bool CHK = decltype(chk_tag)::value;
      float acc[kTI][kTJ];
      // ---- phase A: Y = A X, tanh, dual prox, W = (1 - a^2) p
      if (act) {
        float zL[kTI];
#pragma unroll
        for (int r = 0; r < kTI; ++r) zL[r] = (jt == 0) ? z0[r] : Zb[(jt - 1) * dp + i0 + r];
        tile_product<kTJ>(At, Xs, d, dp, Ns, i0, c0, acc);
#pragma unroll
        for (int r = 0; r < kTI; ++r) {
          const bool row = i0 + r < d;
          float w[kTJ];
#pragma unroll
          for (int c = 0; c < kTJ; ++c) {
            w[c] = 0.f;
            if (row && j0 + c <= N) {
              const float av = tanhf(acc[r][c]);
              const float zl = (c == 0) ? zL[r] : z[r][c - 1];
              const float v = p[r][c] + sig * (z[r][c] - zl);
              const float pn = (HOPF && c == 0 && jt == 0)  // Hopf node 1: prox of sigma g* + lam H
                                   ? __fdividef(v - hc[i0 + r] - lam * av, 1.f + lam + hs[i0 + r])
                                   : (v - lam * av) * ilam;
              if constexpr (CHK) { const float e = pn - p[r][c]; rp += e * e; }
              p[r][c] = pn;
              w[c] = (1.f - av * av) * pn;
            }
          }
          storev<kTJ>(Ws + (size_t)(i0 + r) * Ns + c0, w);
          Pb[jt * dp + i0 + r] = p[r][0];
        }
      }
      group_barrier<G>(grp);
      // ---- phase B: G = A^T W, primal gradient step, relaxation; g-prox of x_0
      if (act) {
        float pR[kTI];
#pragma unroll
        for (int r = 0; r < kTI; ++r)
          pR[r] = (c0 + kTJ < N) ? Pb[(jt + 1) * dp + i0 + r] : 0.f;
        tile_product<kTJ>(Am, Ws, d, dp, Ns, i0, c0, acc);
#pragma unroll
        for (int r = 0; r < kTI; ++r) {
          const int i = i0 + r;
          if (i < d) {
#pragma unroll
            for (int c = 0; c < kTJ; ++c) {
              if (j0 + c < N) {
                const float pn = (c + 1 < kTJ) ? p[r][c + 1 < kTJ ? c + 1 : c] : pR[r];
                const float xo = x[r][c];
                const float xn = xo - tau * (p[r][c] - pn) + taud * acc[r][c];
                if constexpr (CHK) { const float e = xn - xo; rx += e * e; }
                z[r][c] = TH1 ? 2.f * xn - xo : xn + th * (xn - xo);
                x[r][c] = xn;
              }
            }
            if (jt == 0 && !HOPF) {               // x_0 <- prox_{tau g}(x_0 + tau p_1)
              const float xo = x0[r];
              const float xn = (xo + tau * p[r][0] + goff[i]) * ginv[i];
              if constexpr (CHK) { const float e = xn - xo; rx += e * e; }
              z0[r] = TH1 ? 2.f * xn - xo : xn + th * (xn - xo);
              x0[r] = xn;
            }
          }
          storev<kTJ>(Xs + (size_t)i * Ns + c0, x[r]);
          Zb[jt * dp + i] = z[r][kTJ - 1];
        }
      }
      group_barrier<G>(grp);
    };

    int k_it = 0;
    int8_t st = HJ_POINT_MAX_ITER;
    const int max_iter = a.max_iter, check_every = a.check_every;
    while (k_it < max_iter) {
      const int left = max_iter - k_it;
      const int plain = (check_every - 1 < left - 1) ? check_every - 1 : left - 1;
      float dx = 0.f, dpp = 0.f;
      for (int r = 0; r < plain; ++r) step(std::integral_constant<bool, false>{}, dx, dpp);
      float rx = 0.f, rp = 0.f;
      step(std::integral_constant<bool, true>{}, rx, rp);
      k_it += plain + 1;
      // the threads' FP32 partials reduced over each warp in FP32; the group's
      // warp sums accumulated as double-floats (as accurate as FP64, on the
      // FP32 pipe) and compared with tol
      const float wx = warp_sum<float>(rx), wp = warp_sum<float>(rp);
      int verdict;                                // 1 converged, 2 non-finite
      if constexpr (G > 1) {
        if (lane == 0) { tred[2 * wig] = wx; tred[2 * wig + 1] = wp; }
        group_barrier<G>(grp);
        verdict = stop_verdict_g<G, float>(a, tred);
        group_barrier<G>(grp);                    // tred is free for the next test
      } else {
        verdict = stop_verdict1<float>(a, wx, wp);
      }
      if (verdict == 2) { st = HJ_POINT_NONFINITE; break; }
      if (verdict == 1) { st = HJ_POINT_CONVERGED; break; }
    }

    // ---- value: g(x_0) + sum_j <p_j, x_j - x_{j-1}> - delta sum_j H(x_j, p_j); FP32
    // terms (A x from the FP32 copy of A), FP64 sum.  Xs holds the final x.
    double vacc = 0.0;
    if (act) {
      float acc[kTI][kTJ];
      tile_product<kTJ>(At, Xs, d, dp, Ns, i0, c0, acc);
#pragma unroll
      for (int r = 0; r < kTI; ++r) {
        const int i = i0 + r;
        if (i < d) {
          const float xl0 = (jt == 0) ? x0[r] : Xs[(size_t)i * Ns + c0 - 1];
#pragma unroll
          for (int c = 0; c < kTJ; ++c) {
            if (j0 + c <= N) {
              const float pv = p[r][c];
              const float dxv = x[r][c] - ((c == 0) ? xl0 : x[r][c > 0 ? c - 1 : 0]);
              vacc += (double)(pv * dxv - delta_t * (pv * tanhf(acc[r][c]) + 0.5f * pv * pv));
            }
          }
          if (jt == 0) {
            if (HOPF) {                           // -g*(p_1)
              const double p1 = (double)p[r][0];
              vacc -= p1 * a.c[i] + 0.5 * p1 * p1 / a.W2[i];
            } else {
              const double e = (double)x0[r] - a.c[i];
              vacc += 0.5 * a.W2[i] * e * e;
            }
          }
        }
      }
    }
    vacc = warp_sum<double>(vacc);
    if constexpr (G > 1) {
      if (lane == 0) vred[wig] = vacc;
      group_barrier<G>(grp);
      vacc = 0.0;
#pragma unroll
      for (int w = 0; w < G; ++w) vacc += vred[w];
    }
    if (t == 0) {
      a.V[b] = vacc;
      a.iters[b] = k_it;
      a.status[b] = st;
      count_iterations(a, k_it);
    }
    if (act) {
#pragma unroll
      for (int r = 0; r < kTI; ++r) {
        const int i = i0 + r;
        if (i >= d) continue;
#pragma unroll
        for (int c = 0; c < kTJ; ++c) {
          const int j = j0 + c;
          if (j <= N) {
            if (a.traj_x != nullptr) a.traj_x[ref.traj + (size_t)j * d + i] = x[r][c];
            if (a.traj_p != nullptr) a.traj_p[ref.traj + (size_t)j * d + i] = p[r][c];
          }
        }
        if (jt == 0) {
          if (a.traj_x != nullptr)                // Hopf: x_0 = grad g*(p_1) = c + p_1 / W^2
            a.traj_x[ref.traj + i] = HOPF ? (float)(a.c[i] + (double)p[r][0] / a.W2[i]) : x0[r];
          if (a.traj_p != nullptr) a.traj_p[ref.traj + i] = 0.f;
        }
      }
    }
  }
}

template <int TJ, int G, bool TH1, bool HOPF>
hj_status launch_g(const SolveArgs<float>& a, int M, size_t smem, cudaStream_t s) {
  auto kern = lax_td_tile_kernel<TJ, G, TH1, HOPF>;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HJ_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HJ_ERR_CUDA;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return HJ_ERR_CUDA;
  const int threads = 32 * G * M;
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, threads, smem) != cudaSuccess)
    return HJ_ERR_CUDA;
  if (bps < 1) return HJ_ERR_UNSUPPORTED;
  const int64_t ctas_needed = (a.B + M - 1) / M;
  const int64_t cap = (int64_t)bps * nsm;
  const int grid = (int)(ctas_needed < cap ? ctas_needed : cap);
  kern<<<grid, threads, smem, s>>>(a, M);
  return cudaGetLastError() == cudaSuccess ? HJ_OK : HJ_ERR_CUDA;
}

template <int TJ, bool TH1, bool HOPF>
hj_status launch_tj(const SolveArgs<float>& a, int G, int M, size_t smem, cudaStream_t s) {
  if (G == 1) return launch_g<TJ, 1, TH1, HOPF>(a, M, smem, s);
  if (G == 2) return launch_g<TJ, 2, TH1, HOPF>(a, M, smem, s);
  if (G == 4) return launch_g<TJ, 4, TH1, HOPF>(a, M, smem, s);
  if (G == 8) return launch_g<TJ, 8, TH1, HOPF>(a, M, smem, s);
  if constexpr (TJ == 4) {           // 16 warps: four-node tiles only (128 registers)
    if (G == 16) return launch_g<TJ, 16, TH1, HOPF>(a, M, smem, s);
  }
  return HJ_ERR_UNSUPPORTED;
}

// warps per point: a power of two up to 8 (eight-node tiles, about 240
// registers) or 16 (four-node tiles, 128 registers); 0 if it does not fit
int group_warps(int d, int N, int TJ) {
  const int w = (tile_slots(d, N, TJ) + 31) / 32;
  const int g = w <= 1 ? 1 : w <= 2 ? 2 : w <= 4 ? 4 : w <= 8 ? 8 : w <= 16 ? 16 : 0;
  return (g == 16 && TJ != 4) ? 0 : g;
}

// time nodes per tile: 4 where d <= 64 (four-node tiles hold twice the warps
// per SM), else 8
int tile_nodes(int d, int N) {
  const int g4 = group_warps(d, N, 4);
  return (d <= 64 && g4 >= 1) ? 4 : 8;
}

}  // namespace

// Warps per point of the register-tiled kernel for (d, N), 0 when it does not apply.
int td_tile_group_warps(int d, int N) {
  if (d < 1 || d > kMaxD || N < 1 || N > kMaxN) return 0;
  return group_warps(d, N, tile_nodes(d, N));
}

// Runs the register-tiled kernel when it applies (FP32, tanh drift, a point in
// at most 8 warps, shared memory within the opt-in limit); HJ_ERR_UNSUPPORTED
// otherwise, and the caller takes the shared-memory kernel.
hj_status launch_td_tile_solver(const SolveArgs<float>& a, cudaStream_t s) {
  if (a.inner_steps != 1 || a.A == nullptr || a.At == nullptr) return HJ_ERR_UNSUPPORTED;
  const int G = td_tile_group_warps(a.d, a.N);
  if (G == 0) return HJ_ERR_UNSUPPORTED;
  const int TJ = tile_nodes(a.d, a.N);
  int dev = 0, max_optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HJ_ERR_CUDA;
  if (cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
      cudaSuccess)
    return HJ_ERR_CUDA;
  auto bytes = [&](int m) {
    return TJ == 4 ? TileLayout<4>(a.d, a.N, G, m).bytes(m) : TileLayout<8>(a.d, a.N, G, m).bytes(m);
  };
  int M = G == 1 ? 4 : G == 2 ? 2 : 1;
  size_t smem = bytes(M);
  while (M > 1 && smem > (size_t)max_optin) {
    M /= 2;
    smem = bytes(M);
  }
  if (smem > (size_t)max_optin) return HJ_ERR_UNSUPPORTED;
  const bool th1 = a.theta == 1.0;
  const bool hopf = a.formulation == HJ_FORM_HOPF;
  if (TJ == 4) {                     // d <= 32: G is 1 or 2
    if (hopf) return th1 ? launch_tj<4, true, true>(a, G, M, smem, s) : launch_tj<4, false, true>(a, G, M, smem, s);
    return th1 ? launch_tj<4, true, false>(a, G, M, smem, s) : launch_tj<4, false, false>(a, G, M, smem, s);
  }
  if (hopf) return th1 ? launch_tj<8, true, true>(a, G, M, smem, s) : launch_tj<8, false, true>(a, G, M, smem, s);
  return th1 ? launch_tj<8, true, false>(a, G, M, smem, s) : launch_tj<8, false, false>(a, G, M, smem, s);
}

}  // namespace hj
