// Register-resident batched PDHG for the Lax saddle problem (Algorithm 1).
//
// A group of G warps solves one query point at a time.  Lane gl (0..32G-1)
// of the group owns the time nodes j = 1 + gl*NPL .. gl*NPL + NPL (those <= N),
// with x_j, p_j and the relaxed z_j in registers; node 0 (x_0, the g-prox
// node) is spread over lanes 0..D-1, one coordinate each.  The nearest-neighbour terms of the difference
// operator D ((Dz)_j = z_j - z_{j-1}, (D^T p)_j = p_j - p_{j+1}, Appendix A.1)
// cross a lane boundary once per direction and iteration through one
// shared-memory slot per lane (the z of its last node, the p of its first),
// written and read as 16-byte vectors around a group barrier (__syncwarp when
// G = 1).
// Groups draw points from a work counter until the batch is exhausted
// (persistent grid sized to the SM count).
//
// One iteration, per owned node (Section 5.3 updates, loop of Algorithm A.1):
//   ctx  <- H quantities at x_j^k
//   p_j  <- prox_{sigma delta H(x_j^k, .)}(p_j + sigma (z_j - z_{j-1}))     j = 1..N
//   x_0  <- prox_{tau g}(x_0 + tau p_1)
//   x_j  <- x_j - tau (p_j - p_{j+1}) + tau delta grad_x H(x_j^k, p_j)      j = 1..N-1
//   z_j  <- x_j^{k+1} + theta (x_j^{k+1} - x_j^k)
// and, on test iterations, the squared increments: each lane's partial in the
// iterate type, reduced over the warp by shuffles in that type, then
// accumulated over the group's warps (FP32 iterates: as double-floats, as
// accurate as FP64 on the FP32 pipe; FP64: in FP64) and compared with tol.
//
// MIX = true runs the forward-Euler and trapezoid schemes (HJ_SCHEME_FE/TRAP):
// H on interval j is wR H(x_j, .) + wL H(x_{j-1}, .), so the dual step also
// needs x_{j-1}^k (one more exchange slot per lane, and x_0^k as a whole vector),
// x_j's gradient step adds wL grad_x H(x_j, p_{j+1}), and the x_0 step adds
// wL grad_x H(x_0, p_1) before the prox of g.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "families.cuh"
#include "hj_internal.cuh"

namespace hj {

constexpr int kWarpsPerCtaG1 = 4;   // independent single-warp groups per CTA when G = 1

// G = 0 stands for half a warp: two independent 16-lane groups per warp, for
// N <= 16, where a whole warp per point would leave half its lanes without a node.
template <int G>
constexpr int warp_block_threads() { return (G <= 1 ? kWarpsPerCtaG1 : G) * 32; }
template <int G>
constexpr int group_lanes() { return G == 0 ? 16 : 32 * G; }
template <int G>
constexpr int groups_per_cta() { return G == 0 ? 2 * kWarpsPerCtaG1 : (G == 1 ? kWarpsPerCtaG1 : 1); }

// Coordinates padded to a whole number of 16-byte vectors.
template <typename T, int D>
constexpr int padded_dim() { return ((D * (int)sizeof(T) + 15) / 16) * 16 / (int)sizeof(T); }

// Per-CTA shared memory: the family's data, the g-prox of x_0
// (x_0 <- (v + tau W^2 c) / (1 + tau W^2) as offset and reciprocal), the
// per-lane exchange slots of the CTA's groups, and for G > 1 the reduction
// scratch of the CTA's one group.
template <typename T, class F, int D, int G, bool MIX = false, bool HOPF = false>
struct WarpShared {
  static constexpr int kGroups = groups_per_cta<G>();
  static constexpr int kL = group_lanes<G>();
  static constexpr int DP = padded_dim<T, D>();
  typename F::Shared fam;
  alignas(16) T g_off[DP];
  alignas(16) T g_inv[DP];
  alignas(16) T hs[DP];                    // Hopf form: sigma / W^2 and sigma c (node-1 prox)
  alignas(16) T hc[DP];
  double w2d[D], cd[D];
  alignas(16) T zs[kGroups][kL][DP];       // z (in the epilogue x) of each lane's last node
  alignas(16) T ps[kGroups][kL][DP];       // p of each lane's first node
  alignas(16) T x0s[kGroups][DP];          // z_0 (in the epilogue x_0), one coordinate per lane
  // MIX only: x^k of each lane's last node, and x_0^k
  alignas(16) T xs[MIX ? kGroups : 1][MIX ? kL : 1][MIX ? DP : 1];
  alignas(16) T x0x[MIX ? kGroups : 1][MIX ? DP : 1];
  // MIX only: grad_x H(x_0^k, p_1^{k+1}) for the x_0 step, from node 1's lane
  alignas(16) T g0s[MIX ? kGroups : 1][MIX ? DP : 1];
  // Hopf form, families with a tabled node-1 prox: per group, [0] the plain
  // nodes' and [1] node 1's row offsets and row reciprocals (set per point)
  alignas(16) T htab[HOPF ? kGroups : 1][2][2][HOPF ? DP : 1];
  T red[G > 0 ? G : 1][2];
  double vred[G > 0 ? G : 1];
  unsigned long long item;
};

// whether the family's Hopf node-1 prox runs from per-lane tables (F::kHopfTable):
// every lane then takes the same code path, node 1 only other table values
template <class F, class = void>
struct hopf_table : std::false_type {};
template <class F>
struct hopf_table<F, std::void_t<decltype(F::kHopfTable)>>
    : std::integral_constant<bool, F::kHopfTable> {};

// lanes of this thread's 16-lane half
__device__ __forceinline__ unsigned half_mask() { return 0xFFFFu << (threadIdx.x & 16); }

template <int G>
__device__ __forceinline__ void group_sync() {
  if constexpr (G > 1) __syncthreads();
  else if constexpr (G == 1) __syncwarp();
  else __syncwarp(half_mask());
}

// sum over the lanes of a warp, or of a half warp for G = 0
template <int G, typename U>
__device__ __forceinline__ U lanes_sum(U v) {
  if constexpr (G == 0) {
    const unsigned m = half_mask();
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o);
    return v;
  } else {
    return warp_sum<U>(v);
  }
}

// 16-byte vector copies between a D-array in registers and a padded slot.
template <typename T, int D>
__device__ __forceinline__ void slot_store(T* dst, const T (&v)[D]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int k = 0; k + 4 <= D; k += 4)
      *reinterpret_cast<float4*>(dst + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
#pragma unroll
    for (int k = D - D % 4; k < D; ++k) dst[k] = v[k];
  } else {
#pragma unroll
    for (int k = 0; k + 2 <= D; k += 2)
      *reinterpret_cast<double2*>(dst + k) = make_double2(v[k], v[k + 1]);
#pragma unroll
    for (int k = D - D % 2; k < D; ++k) dst[k] = v[k];
  }
}

template <typename T, int D>
__device__ __forceinline__ void slot_load(const T* src, T (&v)[D]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int k = 0; k + 4 <= D; k += 4) {
      const float4 q = *reinterpret_cast<const float4*>(src + k);
      v[k] = q.x; v[k + 1] = q.y; v[k + 2] = q.z; v[k + 3] = q.w;
    }
#pragma unroll
    for (int k = D - D % 4; k < D; ++k) v[k] = src[k];
  } else {
#pragma unroll
    for (int k = 0; k + 2 <= D; k += 2) {
      const double2 q = *reinterpret_cast<const double2*>(src + k);
      v[k] = q.x; v[k + 1] = q.y;
    }
#pragma unroll
    for (int k = D - D % 2; k < D; ++k) v[k] = src[k];
  }
}

// H quantities of node j at its time s_j = j delta (time-dependent families)
template <class F, typename T, int D>
__device__ __forceinline__ void node_context(const F& fam, const T (&x)[D], T sj,
                                             typename F::Ctx& c) {
  if constexpr (F::kTimeDep) fam.context_t(x, sj, c);
  else fam.context(x, c);
}
template <class F, typename T, int D>
__device__ __forceinline__ T node_Ht(const F& fam, const T (&x)[D], const T (&p)[D], T sj) {
  if constexpr (F::kTimeDep) return fam.Ht_t(x, p, sj);
  else return fam.Ht(x, p);
}
template <class F, typename T, int D>
__device__ __forceinline__ double node_H64(const F& fam, const T (&x)[D], const T (&p)[D],
                                           double sj) {
  if constexpr (F::kTimeDep) return fam.H64_t(x, p, sj);
  else return fam.H64(x, p);
}

// relaxation z = x_new + theta (x_new - x); TH1: theta = 1 (the paper's choice,
// Section 6), one fused multiply-add per coordinate
template <typename T, bool TH1>
__device__ __forceinline__ T relax(T xn, T xo, T th) {
  if constexpr (TH1) return T(2) * xn - xo;
  else return xn + th * (xn - xo);
}

template <typename T, class F, int D, int NPL, int G, bool TH1, bool HOPF, bool MIX>
__device__ __forceinline__ void solve_point(const SolveArgs<T>& a, const F& fam, int64_t item,
                                            int lane, int wg, WarpShared<T, F, D, G, MIX, HOPF>& sh) {
  static_assert(!(MIX && HOPF), "the mixed schemes are Lax-form problems");
  const PointRef<T> pt = point_ref(a, item);
  const int N = pt.N;
  const int gl = wg * 32 + lane;              // lane: 0..15 for G = 0
  if (N < 1 || N > group_lanes<G>() * NPL) {  // the host never routes such a point here
    if (gl == 0) { a.status[pt.id] = HJ_POINT_INVALID; a.iters[pt.id] = 0; a.V[pt.id] = 0.0; }
    return;
  }
  // iteration constants in the iterate type only (delta = t / N)
  const T sig = a.sigma_t, tau = a.tau_t, th = a.theta_t;
  const T delta_t = T(a.t[pt.id]) / T(N);
  const T lam = sig * delta_t, taud = tau * delta_t;
  const T wr = a.mix_wr_t, wl = a.mix_wl_t;      // MIX: weights of H at x_j and x_{j-1}
  const typename F::PC pc = fam.point(lam);
  const uint64_t gid = (uint64_t)(a.point_offset + pt.id);
  if constexpr (HOPF && hopf_table<F>::value) {
    // this point's row tables (read after the first iteration's group barrier)
    const int tg = (G == 1) ? (int)(threadIdx.x >> 5) : (G == 0 ? (int)(threadIdx.x >> 4) : 0);
    constexpr int TDP = WarpShared<T, F, D, G, MIX, HOPF>::DP;
    for (int k = gl; k < TDP; k += group_lanes<G>()) {
      T op = T(0), dp = T(0), of = T(0), df = T(0);
      if (k < D) fam.hopf_row(pc, sh.hs, sh.hc, k, op, dp, of, df);
      sh.htab[tg][0][0][k] = op; sh.htab[tg][0][1][k] = dp;
      sh.htab[tg][1][0][k] = of; sh.htab[tg][1][1][k] = df;
    }
  }

  T x[NPL][D], p[NPL][D], z[NPL][D];
  // x_0: lane gl < D holds coordinate gl (x0 = x_0[gl], z0 = z_0[gl])
  const bool own0 = gl < D;
  const int k0 = own0 ? gl : 0;
  T x0 = T(0), z0 = T(0);
  const T goff = sh.g_off[k0], ginv = sh.g_inv[k0];
  const int jbase = 1 + gl * NPL;
  {
    if (a.warm_x == nullptr) {
      const InitGuess<T> ig(a.radius);
#pragma unroll
      for (int i = 0; i < NPL; ++i) {
        const int j = jbase + i;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const double xq = pt.xq[k];
          T xv = T(0), pv = T(0);
          if (j < N) xv = ig.x(xq, a.seed, gid, j, k);
          else if (j == N) xv = T(xq);
          if (j <= N) pv = ig.p(a.seed, gid, j, k);
          x[i][k] = xv; p[i][k] = pv; z[i][k] = xv;
        }
      }
      if (own0 && !HOPF) x0 = ig.x(pt.xq[k0], a.seed, gid, 0, k0);
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
          else if (j == N) xv = T(pt.xq[k]);
          if (j <= N) pv = T(a.cost_sign) * wp[(size_t)j * D + k];   // traj_p convention
          x[i][k] = xv; p[i][k] = pv; z[i][k] = xv;
        }
      }
      if (own0 && !HOPF) x0 = wx[k0];
    }
    z0 = x0;
  }
  const int grp = (G == 1) ? (int)(threadIdx.x >> 5) : (G == 0 ? (int)(threadIdx.x >> 4) : 0);
  T* zslot = &sh.zs[grp][0][0];
  T* pslot = &sh.ps[grp][0][0];
  T* x0slot = &sh.x0s[grp][0];
  if (own0) x0slot[k0] = z0;                  // read by lane 0 after the first barrier
  T* xslot = &sh.xs[grp][0][0];
  T* x0xslot = &sh.x0x[grp][0];
  T* g0slot = &sh.g0s[grp][0];
  if constexpr (MIX) { if (own0) x0xslot[k0] = x0; }
  constexpr int DP = WarpShared<T, F, D, G, MIX, HOPF>::DP;
  constexpr int kLanes = group_lanes<G>();

  // One iteration; CHK adds the squared increments (test iterations only, so
  // the plain iterations carry no residual code at all).
  // On test iterations with the value test on (value_tol > 0, Lax form,
  // backward Euler) vacc collects this lane's part of fval at (x^{k+1}, p^{k+1})
  // in the summed-by-parts form
  //   g(x_0) - <p_1, x_0> + sum_{j<N} <p_j - p_{j+1}, x_j> + <p_N, x_N> - delta sum_j H(x_j, p_j)
  // (for the game the q-pairings enter with the opposite sign).
  constexpr bool kValueTest = !MIX && !HOPF;
  auto coord_sign = [&](int k) -> T {
    if constexpr (F::kGame) return k < fam.d1 ? T(1) : T(-1);
    else return T(1);
  };
  auto step = [&](auto chk_tag, T& rx, T& rp, T& vacc) {
    constexpr bool CHK = decltype(chk_tag)::value;
    typename F::Ctx ctx[NPL];
    // ---- z_{j-1} of the first owned node: the left lane's slot (z^k of its last node)
    slot_store<T, D>(zslot + gl * DP, z[NPL - 1]);
    if constexpr (MIX) slot_store<T, D>(xslot + gl * DP, x[NPL - 1]);
    group_sync<G>();
    T zl[D];
    slot_load<T, D>(gl > 0 ? zslot + (gl - 1) * DP : x0slot, zl);
    // MIX: x_{j-1}^k of the first owned node and its H quantities; x_0^k whole
    // (read here, before the next barrier, since the x_0 step rewrites its slot)
    [[maybe_unused]] T xlv[MIX ? D : 1];
    [[maybe_unused]] T x0v[MIX ? D : 1];
    [[maybe_unused]] typename F::Ctx ctxl;
    if constexpr (MIX) {
      slot_load<T, D>(gl > 0 ? xslot + (gl - 1) * DP : x0xslot, xlv);
      if (own0) slot_load<T, D>(x0xslot, x0v);
      fam.context(xlv, ctxl);
    }
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
      if (jbase + i <= N) {
        node_context(fam, x[i], T(jbase + i) * delta_t, ctx[i]);
        T v[D], dz[D];
        if (i == 0) v_sub<T, D>(dz, z[i], zl);
        else v_sub<T, D>(dz, z[i], z[i > 0 ? i - 1 : 0]);
        v_fma<T, D>(v, sig, dz, p[i]);                       // p + sigma (z_j - z_{j-1})
        if constexpr (HOPF) {                                // Hopf: node 1 also carries g*
          if constexpr (hopf_table<F>::value) {
            const T* tb = &sh.htab[grp][(i == 0 && gl == 0) ? 1 : 0][0][0];
            fam.prox_hopf(ctx[i], pc, x[i], v, tb, tb + DP);
          } else {
            if (i == 0 && gl == 0) fam.prox_first(ctx[i], pc, x[i], v, sh.hs, sh.hc);
            else fam.prox(ctx[i], pc, x[i], v);
          }
        } else if constexpr (MIX) {                          // prox of lam (wR H(x_j) + wL H(x_{j-1}))
          if (i == 0) fam.prox_mix(ctx[i], ctxl, pc, wr, wl, x[i], xlv, v);
          else fam.prox_mix(ctx[i], ctx[i > 0 ? i - 1 : 0], pc, wr, wl, x[i], x[i > 0 ? i - 1 : 0], v);
        } else {
          fam.prox(ctx[i], pc, x[i], v);
        }
        if constexpr (CHK) {
          T e[D];
          v_sub<T, D>(e, v, p[i]);
          rp += v_sumsq<T, D>(e);
        }
#pragma unroll
        for (int k = 0; k < D; ++k) p[i][k] = v[k];
      }
    }
    // MIX (not the game): node 1's lane holds x_0^k's context (its left
    // neighbour's) and p_1^{k+1}: it forms grad_x H(x_0^k, p_1) once for the
    // x_0 lanes, which read it after the barrier below
    if constexpr (MIX && !F::kGame && F::kHasGradX) {
      if (gl == 0) {
        T g0[D];
        fam.gradx(ctxl, xlv, p[0], g0);
        slot_store<T, D>(g0slot, g0);
      }
    }
    // ---- primal step: p_{j+1} of the last owned node from the right lane's slot
    slot_store<T, D>(pslot + gl * DP, p[0]);
    group_sync<G>();
    T pr[D];
    if (gl + 1 < kLanes) {
      slot_load<T, D>(pslot + (gl + 1) * DP, pr);
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) pr[k] = T(0);    // the last lane never updates an x with it
    }
    if (own0 && !HOPF) {
      // x_0 <- prox_{tau g}(x_0 + tau p_1), coordinate k0; p_1 is lane 0's slot
      T xn;
      if constexpr (MIX && F::kGame) {
        // the whole node-0 step in every x_0 lane (the y-block needs all of x_0^{k+1})
        T p1[D], zn0[D];
        slot_load<T, D>(pslot, p1);
        fam.node0_step_mix(x0v, p1, tau, taud * wl, sh.g_off, sh.g_inv, zn0);
        xn = T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) xn = (k == k0) ? zn0[k] : xn;
      } else {
        T v0 = x0 + tau * pslot[k0];                          // (D^T p)_0 = -p_1
        if constexpr (MIX) {
          // + tau delta wL grad_x H(x_0^k, p_1), coordinate k0 (from node 1's lane)
          if constexpr (F::kHasGradX) v0 += taud * wl * g0slot[k0];
        }
        xn = (v0 + goff) * ginv;
      }
      if constexpr (CHK) { const T e = xn - x0; rx += e * e; }
      if constexpr (CHK && kValueTest) {
        if (a.value_stop) {                              // g(x_0) - <p_1, x_0>, coordinate k0
          const T e = xn - T(sh.cd[k0]);
          vacc += T(0.5) * T(sh.w2d[k0]) * e * e - coord_sign(k0) * pslot[k0] * xn;
        }
      }
      z0 = relax<T, TH1>(xn, x0, th);
      x0 = xn;
      x0slot[k0] = z0;
      if constexpr (MIX) x0xslot[k0] = xn;
    }
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
      if (jbase + i < N) {
        T xn[D], dp[D];
        if (i == NPL - 1) v_sub<T, D>(dp, p[i], pr);
        else v_sub<T, D>(dp, p[i], p[i + 1 < NPL ? i + 1 : i]);
        v_fma<T, D>(xn, -tau, dp, x[i]);                     // x - tau (p_j - p_{j+1})
        if constexpr (F::kGame && MIX) {
          // norms of the two costates weighted: wR at P_j, wL at P_{j+1}
          T np1, nq1, np2, nq2;
          fam.norms(p[i], np1, nq1);
          if (i == NPL - 1) fam.norms(pr, np2, nq2);
          else fam.norms(p[i + 1 < NPL ? i + 1 : i], np2, nq2);
          fam.game_step_norms(ctx[i], x[i], wr * np1 + wl * np2, wr * nq1 + wl * nq2, taud, xn);
        } else if constexpr (F::kGame) {
          fam.game_step(ctx[i], x[i], p[i], taud, xn);      // descent in x, ascent in y
        } else if constexpr (MIX) {
          // + tau delta (wR grad_x H(x_j, p_j) + wL grad_x H(x_j, p_{j+1}))
          T g[D], g2[D];
          fam.gradx(ctx[i], x[i], p[i], g);
          if (i == NPL - 1) fam.gradx(ctx[i], x[i], pr, g2);
          else fam.gradx(ctx[i], x[i], p[i + 1 < NPL ? i + 1 : i], g2);
#pragma unroll
          for (int k = 0; k < D; ++k) g[k] = wr * g[k] + wl * g2[k];
          T base[D];
#pragma unroll
          for (int k = 0; k < D; ++k) base[k] = xn[k];
          v_fma<T, D>(xn, taud, g, base);
        } else if (F::kHasGradX) {
          T g[D];
          fam.gradx(ctx[i], x[i], p[i], g);
          T base[D];
#pragma unroll
          for (int k = 0; k < D; ++k) base[k] = xn[k];
          v_fma<T, D>(xn, taud, g, base);                    // + tau delta grad_x H
          for (int s = 1; s < a.inner_steps; ++s) {
            typename F::Ctx c2;
            node_context(fam, xn, T(jbase + i) * delta_t, c2);
            fam.gradx(c2, xn, p[i], g);
            v_fma<T, D>(xn, taud, g, base);
          }
        }
        if constexpr (CHK) {
          T e[D];
          v_sub<T, D>(e, xn, x[i]);
          rx += v_sumsq<T, D>(e);
        }
        if constexpr (CHK && kValueTest) {
          if (a.value_stop) {                            // <p_j - p_{j+1}, x_j> - delta H(x_j, p_j)
            T s = T(0);
#pragma unroll
            for (int k = 0; k < D; ++k) s += coord_sign(k) * dp[k] * xn[k];
            vacc += s - delta_t * node_Ht(fam, xn, p[i], T(jbase + i) * delta_t);
          }
        }
        if constexpr (TH1) {
          v_fms<T, D>(z[i], T(2), xn, x[i]);                // z = 2 x_new - x
        } else {
#pragma unroll
          for (int k = 0; k < D; ++k) z[i][k] = relax<T, TH1>(xn[k], x[i][k], th);
        }
#pragma unroll
        for (int k = 0; k < D; ++k) x[i][k] = xn[k];
      } else if (jbase + i == N) {
        if constexpr (CHK && kValueTest) {
          if (a.value_stop) {                            // <p_N, x_N> - delta H(x_N, p_N)
            T s = T(0);
#pragma unroll
            for (int k = 0; k < D; ++k) s += coord_sign(k) * p[i][k] * x[i][k];
            vacc += s - delta_t * node_Ht(fam, x[i], p[i], T(jbase + i) * delta_t);
          }
        }
      }
    }
  };

  // Test after every check_every-th iteration and after iteration max_iter.
  int k_it = 0;
  int8_t st = HJ_POINT_MAX_ITER;
  double vprev = 0.0;                                // fval at the previous test
  bool have_prev = false;
  const int max_iter = a.max_iter, check_every = a.check_every;
  while (k_it < max_iter) {
    const int left = max_iter - k_it;
    const int plain = (check_every - 1 < left - 1) ? check_every - 1 : left - 1;
    T dummy_x = T(0), dummy_p = T(0), dummy_v = T(0);
    for (int r = 0; r < plain; ++r)
      step(std::integral_constant<bool, false>{}, dummy_x, dummy_p, dummy_v);
    T rx = T(0), rp = T(0), vacc = T(0);
    step(std::integral_constant<bool, true>{}, rx, rp, vacc);
    k_it += plain + 1;
    // each lane's partial (its own nodes, in the iterate type) reduced over the
    // warp by shuffles in that type (a 5-level tree: relative error <= 5 ulp);
    // the group's warp sums accumulated as double-floats (stop_verdict: as
    // accurate as FP64, on the FP32 pipe) and compared with tol
    const T wx = lanes_sum<G, T>(rx), wp = lanes_sum<G, T>(rp);
    int verdict;                                     // 1 converged, 2 non-finite
    if constexpr (G > 1) {
      if (lane == 0) { sh.red[wg][0] = wx; sh.red[wg][1] = wp; }
      __syncthreads();
      verdict = stop_verdict_g<G, T>(a, &sh.red[0][0]);
    } else {
      verdict = stop_verdict1<T>(a, wx, wp);
    }
    if (verdict == 2) { st = HJ_POINT_NONFINITE; break; }
    if (verdict == 1) { st = HJ_POINT_CONVERGED; break; }
    if constexpr (kValueTest) {
      if (a.value_stop) {                 // the value moved less than value_tol since the last test
        double v = lanes_sum<G, double>((double)vacc);
        if constexpr (G > 1) {
          if (lane == 0) sh.vred[wg] = v;
          __syncthreads();
          v = 0.0;
#pragma unroll
          for (int w = 0; w < G; ++w) v += sh.vred[w];
          __syncthreads();                // every warp has read before the next write
        }
        if (have_prev && fabs(v - vprev) < a.value_tol) { st = HJ_POINT_VALUE_STOP; break; }
        vprev = v;
        have_prev = true;
      }
    }
  }

  // ---- value (fval of Algorithm 1), summed in FP64, and outputs
  group_sync<G>();                                 // every lane is done with the slots
  slot_store<T, D>(zslot + gl * DP, x[NPL - 1]);
  if (own0) x0slot[k0] = x0;
  group_sync<G>();
  double acc = 0.0;
  {
    const double delta = a.t[pt.id] / N;
    T xl[D];
    slot_load<T, D>(gl > 0 ? zslot + (gl - 1) * DP : x0slot, xl);
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
      if (jbase + i <= N) {
        if constexpr (sizeof(T) == 4) {
          // FP32 iterates: each node's term <p_j, x_j - x_{j-1}> - delta H(x_j, p_j)
          // in FP32, the sum over nodes in FP64
          T s = T(0);
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const T term = p[i][k] * (x[i][k] - ((i == 0) ? xl[k] : x[i - 1][k]));
            if constexpr (F::kGame) s += (k < fam.d1) ? term : -term;   // <p, dx> - <q, dy>
            else s += term;
          }
          if constexpr (MIX) {
            const T hl = (i == 0) ? fam.Ht(xl, p[i]) : fam.Ht(x[i > 0 ? i - 1 : 0], p[i]);
            acc += (double)(s - delta_t * (wr * fam.Ht(x[i], p[i]) + wl * hl));
          } else {
            acc += (double)(s - delta_t * node_Ht(fam, x[i], p[i], T(jbase + i) * delta_t));
          }
        } else {
          double s = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const double xm = (double)((i == 0) ? xl[k] : x[i - 1][k]);
            const double term = (double)p[i][k] * ((double)x[i][k] - xm);
            if constexpr (F::kGame) s += (k < fam.d1) ? term : -term;
            else s += term;
          }
          if constexpr (MIX) {
            const double hl = (i == 0) ? fam.H64(xl, p[i]) : fam.H64(x[i > 0 ? i - 1 : 0], p[i]);
            acc += s - delta * (a.mix_wr * fam.H64(x[i], p[i]) + a.mix_wl * hl);
          } else {
            acc += s - delta * node_H64(fam, x[i], p[i], (double)(jbase + i) * delta);
          }
        }
      }
    }
    if (own0) {
      if constexpr (HOPF) {                           // -g*(p_1), coordinate k0 (x_0 = 0 above)
        const double p1 = (double)pslot[k0];
        acc -= p1 * sh.cd[k0] + 0.5 * p1 * p1 / sh.w2d[k0];
      } else {
        const double e = (double)x0 - sh.cd[k0];
        acc += 0.5 * sh.w2d[k0] * e * e;              // g(x_0), coordinate k0
      }
    }
  }
  acc = lanes_sum<G, double>(acc);
  if constexpr (G > 1) {
    if (lane == 0) sh.vred[wg] = acc;
    __syncthreads();
    acc = 0.0;
#pragma unroll
    for (int w = 0; w < G; ++w) acc += sh.vred[w];
  }
  if (gl == 0) {
    a.V[pt.id] = a.cost_sign * acc;
    a.iters[pt.id] = k_it;
    a.status[pt.id] = st;
    count_iterations(a, k_it);
  }
  if (a.traj_x != nullptr) {
    T* o = a.traj_x + pt.traj;
#pragma unroll
    for (int i = 0; i < NPL; ++i)
      if (jbase + i <= N)
#pragma unroll
        for (int k = 0; k < D; ++k) o[(size_t)(jbase + i) * D + k] = x[i][k];
    if (own0) o[k0] = HOPF ? T(sh.cd[k0] + (double)pslot[k0] / sh.w2d[k0]) : x0;
  }
  if (a.traj_p != nullptr) {
    T* o = a.traj_p + pt.traj;
#pragma unroll
    for (int i = 0; i < NPL; ++i)
      if (jbase + i <= N)
#pragma unroll
        for (int k = 0; k < D; ++k) o[(size_t)(jbase + i) * D + k] = T(a.cost_sign) * p[i][k];
    if (own0) o[k0] = T(0);
  }
}

template <typename T, class F, int D, int NPL, int G, bool TH1, bool HOPF, bool MIX>
__global__ void __launch_bounds__(warp_block_threads<G>())
lax_warp_kernel(const SolveArgs<T> a) {
  __shared__ WarpShared<T, F, D, G, MIX, HOPF> sh;
  F::load_shared(a, sh.fam);
  for (int k = threadIdx.x; k < WarpShared<T, F, D, G, MIX, HOPF>::DP; k += blockDim.x) {
    // cost_sign = -1 (negative eikonal): the positive equation with initial data -g
    const double w2 = k < D ? a.cost_sign * a.W2[k] : 0.0, c = k < D ? a.c[k] : 0.0;
    if (k < D) { sh.w2d[k] = w2; sh.cd[k] = c; }
    // a game's maximising coordinates take the ascent prox of g at y_0: the
    // same formula with -W^2 (the stretch, tau W^2 < 1)
    const double w2p = (F::kGame && k >= a.game_d1) ? -w2 : w2;
    sh.g_off[k] = T(a.tau * w2p * c);
    sh.g_inv[k] = T(1.0 / (1.0 + a.tau * w2p));
    sh.hs[k] = (HOPF && k < D) ? T(a.sigma / w2) : T(0);
    sh.hc[k] = T(a.sigma * c);
  }
  __syncthreads();
  const F fam(a, sh.fam);
  const int lane = (G == 0) ? (int)(threadIdx.x & 15) : (int)(threadIdx.x & 31);
  const int wg = (G <= 1) ? 0 : (int)(threadIdx.x >> 5);
  for (;;) {
    unsigned long long drawn;
    if constexpr (G == 1) {
      unsigned long long bb = 0;
      if (lane == 0) bb = draw_item(a);
      drawn = __shfl_sync(kFull, bb, 0);
    } else if constexpr (G == 0) {           // each half draws its own points
      unsigned long long bb = 0;
      if (lane == 0) bb = draw_item(a);
      drawn = __shfl_sync(half_mask(), bb, (int)(threadIdx.x & 16));
    } else {
      __syncthreads();                       // the previous point is finished by every warp
      if (threadIdx.x == 0) sh.item = draw_item(a);
      __syncthreads();
      drawn = sh.item;
    }
    const int64_t item = (int64_t)drawn;
    if (item >= a.B) break;
    solve_point<T, F, D, NPL, G, TH1, HOPF, MIX>(a, fam, item, lane, wg, sh);
  }
}

template <typename T, class F, int D, int NPL, int G, bool TH1, bool HOPF, bool MIX>
hj_status launch_warp_cfg_th(const SolveArgs<T>& a, cudaStream_t s) {
  static int blocks_per_sm = -1;
  static int num_sms = 0;
  auto kern = lax_warp_kernel<T, F, D, NPL, G, TH1, HOPF, MIX>;
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
  constexpr int points_per_cta = groups_per_cta<G>();
  const int64_t need = (a.B + points_per_cta - 1) / points_per_cta;
  const int64_t cap = (int64_t)blocks_per_sm * num_sms;
  const int grid = (int)(need < cap ? need : cap);
  if (grid <= 0) return HJ_OK;
  kern<<<grid, threads, 0, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? HJ_OK : HJ_ERR_CUDA;
}

// theta = 1 (the paper's choice) gets its own kernel; the mixed schemes run
// the general relaxation z = x + theta (x - x^k) for every theta
template <typename T, class F, int D, int NPL, int G, bool HOPF, bool MIX>
hj_status launch_warp_cfg(const SolveArgs<T>& a, cudaStream_t s) {
  if constexpr (MIX) {
    return launch_warp_cfg_th<T, F, D, NPL, G, false, HOPF, MIX>(a, s);
  } else {
    return a.theta == 1.0 ? launch_warp_cfg_th<T, F, D, NPL, G, true, HOPF, MIX>(a, s)
                          : launch_warp_cfg_th<T, F, D, NPL, G, false, HOPF, MIX>(a, s);
  }
}

// Every (G, NPL) the library instantiates: FP32 G in {1,2,4,8} x NPL in {1,2};
// FP64 G in {1,2,4,8} x NPL = 1; and half-warp groups (G = 0, NPL = 1, N <= 16); the mixed schemes in FP64 stop at G = 4 (their
// second exchange slot would bring the static shared memory of the FP64 G = 8
// group to about 75 KB; that instantiation is not built).
template <typename T, template <typename, int> class F, int D, bool HOPF, bool MIX = false>
hj_status launch_warp_shape(const SolveArgs<T>& a, WarpConfig c, cudaStream_t s) {
  constexpr bool f64 = sizeof(T) == 8;
  if (c.half) {                                  // two 16-lane groups per warp
    if constexpr (D <= 16) {
      if (c.NPL == 1) return launch_warp_cfg<T, F<T, D>, D, 1, 0, HOPF, MIX>(a, s);
    }
    return HJ_ERR_UNSUPPORTED;
  }
  if (c.NPL == 1) {
    switch (c.G) {
      case 1: return launch_warp_cfg<T, F<T, D>, D, 1, 1, HOPF, MIX>(a, s);
      case 2: return launch_warp_cfg<T, F<T, D>, D, 1, 2, HOPF, MIX>(a, s);
      case 4: return launch_warp_cfg<T, F<T, D>, D, 1, 4, HOPF, MIX>(a, s);
      case 8:
        if constexpr (f64 && MIX) return HJ_ERR_UNSUPPORTED;
        else return launch_warp_cfg<T, F<T, D>, D, 1, 8, HOPF, MIX>(a, s);
      default: return HJ_ERR_UNSUPPORTED;
    }
  }
  if constexpr (!f64) {
    if (c.NPL == 2) {
      switch (c.G) {
        case 1: return launch_warp_cfg<T, F<T, D>, D, 2, 1, HOPF, MIX>(a, s);
        case 2: return launch_warp_cfg<T, F<T, D>, D, 2, 2, HOPF, MIX>(a, s);
        case 4: return launch_warp_cfg<T, F<T, D>, D, 2, 4, HOPF, MIX>(a, s);
        case 8: return launch_warp_cfg<T, F<T, D>, D, 2, 8, HOPF, MIX>(a, s);
        default: return HJ_ERR_UNSUPPORTED;
      }
    }
  }
  return HJ_ERR_UNSUPPORTED;
}

}  // namespace hj
