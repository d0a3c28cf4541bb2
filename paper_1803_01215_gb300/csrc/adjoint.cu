// Reverse sweep through the PDHG iterations (the adjoint of Algorithm 1 run for
// exactly K iterations), with the iterates checkpointed every C iterations.
//
// For a point solved in K iterations, V_K = fval(x^K, p^K) (Algorithm 1's value
// at the final iterate) is a smooth function of the cost weights W, the centre
// c, the dynamics parameters and the query point x (through x_N = x and the
// initial guess x^0 = x + r u).  This kernel returns its exact gradient by
// reverse-mode differentiation of the K iterations:
//   forward   run the K iterations again from the counter-based initial guess,
//             storing (x, p, z) at iterations 0, C, 2C, ... in workspace;
//   backward  for k = K-1 .. 0: rebuild s^k from its checkpoint (at most C-1
//             forward steps), then apply the transposed Jacobian of step k to
//             the adjoint (xbar, pbar, zbar), accumulating parameter adjoints.
// At a converged point this equals the envelope gradient of hj_solve_grad.
// One CTA of G warps per point (lane l <-> node l + 1; lane 0 also owns node
// 0); neighbour terms go through per-lane shared-memory slots, as in the solver.
// Families: quadratic (d <= 4) and quadcopter (d = 12).
#include <cuda_runtime.h>

#include "families.cuh"
#include "hj_internal.cuh"
#include "hjpdhg.h"

namespace hj {

namespace {

// ---------------------------------------------------------------- per-node family math
// Quadcopter pieces in the iterate type (the solver's formulas, written out
// with their intermediates so the reverse rules can reuse them).
template <typename T>
struct QCNode {
  T a[3], J[9], H2[27];   // thrust direction, d a / d angles, second derivatives
};

template <typename T>
__device__ __forceinline__ void qc_node(const T (&x)[12], QCNode<T>& n) {
  T sps, cps, sth, cth, sph, cph;
  sin_cos<T>(x[3], &sps, &cps);
  sin_cos<T>(x[4], &sth, &cth);
  sin_cos<T>(x[5], &sph, &cph);
  n.a[0] = sph * sps + cph * cps * sth;
  n.a[1] = -cps * sph + cph * sth * sps;
  n.a[2] = cth * cph;
  // J[3r + c] = d a_r / d angle_c, angles (psi, theta, phi)
  n.J[0] = sph * cps - cph * sps * sth; n.J[1] = cph * cps * cth; n.J[2] = cph * sps - sph * cps * sth;
  n.J[3] = sps * sph + cph * sth * cps; n.J[4] = cph * cth * sps; n.J[5] = -cps * cph - sph * sth * sps;
  n.J[6] = T(0);                        n.J[7] = -sth * cph;       n.J[8] = -cth * sph;
  // H2[9r + 3c + k] = d^2 a_r / d angle_c d angle_k
  T* h = n.H2;
  // a0
  h[0] = -n.a[0];                 h[1] = -cph * sps * cth;        h[2] = cph * cps + sph * sps * sth;
  h[3] = h[1];                    h[4] = -cph * cps * sth;        h[5] = -sph * cps * cth;
  h[6] = h[2];                    h[7] = h[5];                    h[8] = -n.a[0];
  // a1
  h[9] = -n.a[1];                 h[10] = cph * cth * cps;        h[11] = sps * cph - sph * sth * cps;
  h[12] = h[10];                  h[13] = -cph * sth * sps;       h[14] = -sph * cth * sps;
  h[15] = h[11];                  h[16] = h[14];                  h[17] = -n.a[1];
  // a2
  h[18] = T(0); h[19] = T(0); h[20] = T(0);
  h[21] = T(0); h[22] = -n.a[2];  h[23] = sth * sph;
  h[24] = T(0); h[25] = h[23];    h[26] = -n.a[2];
}

struct QCPar { double m, ah, gz, eps; };

// p' = prox(x, v) of the quadcopter H (Sherman-Morrison on rows 6-8)
template <typename T>
__device__ __forceinline__ void qc_prox(const QCNode<T>& n, const QCPar& q, T L, const T (&x)[12],
                                        const T (&v)[12], T (&pp)[12]) {
  const T al = T(1) + L * T(q.eps), ial = T(1) / al, irate = T(1) / (al + L), minv = T(1.0 / q.m);
  for (int k = 0; k < 6; ++k) pp[k] = (v[k] - L * x[6 + k]) * ial;
  for (int k = 9; k < 12; ++k) pp[k] = v[k] * irate;
  T w[3], b[3];
  for (int r = 0; r < 3; ++r) {
    w[r] = v[6 + r] - L * (T(q.ah) * n.a[r] - (r == 2 ? T(q.gz) : T(0)));
    b[r] = n.a[r] * minv;
  }
  const T bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  const T bw = b[0] * w[0] + b[1] * w[1] + b[2] * w[2];
  const T f = L * bw / (al + L * bb);
  for (int r = 0; r < 3; ++r) pp[6 + r] = (w[r] - f * b[r]) * ial;
}

// grad_x H(x, p) of the quadcopter
template <typename T>
__device__ __forceinline__ void qc_gradx(const QCNode<T>& n, const QCPar& q, const T (&p)[12],
                                         T (&g)[12]) {
  const T minv = T(1.0 / q.m);
  const T s = n.a[0] * p[6] + n.a[1] * p[7] + n.a[2] * p[8];
  const T coef = T(q.ah) + s * minv * minv;
  g[0] = g[1] = g[2] = T(0);
  for (int c = 0; c < 3; ++c) g[3 + c] = coef * (n.J[c] * p[6] + n.J[3 + c] * p[7] + n.J[6 + c] * p[8]);
  for (int k = 0; k < 3; ++k) { g[6 + k] = p[k]; g[9 + k] = p[3 + k]; }
}

// grad_p H(x, p) = f0 + B B^T p + eps p
template <typename T>
__device__ __forceinline__ void qc_gradp(const QCNode<T>& n, const QCPar& q, const T (&x)[12],
                                         const T (&p)[12], T (&g)[12]) {
  const T minv = T(1.0 / q.m), e = T(q.eps);
  const T u0 = (n.a[0] * p[6] + n.a[1] * p[7] + n.a[2] * p[8]) * minv;
  for (int k = 0; k < 3; ++k) { g[k] = x[6 + k] + e * p[k]; g[3 + k] = x[9 + k] + e * p[3 + k]; }
  for (int r = 0; r < 3; ++r)
    g[6 + r] = T(q.ah) * n.a[r] - (r == 2 ? T(q.gz) : T(0)) + n.a[r] * minv * u0 + e * p[6 + r];
  for (int k = 9; k < 12; ++k) g[k] = p[k] + e * p[k];
}

// d H / d (m, a_h, g_z, eps) at (x, p)
template <typename T>
__device__ __forceinline__ void qc_dHdpar(const QCNode<T>& n, const QCPar& q, const T (&p)[12],
                                          double (&o)[4]) {
  const double s = (double)(n.a[0] * p[6] + n.a[1] * p[7] + n.a[2] * p[8]);
  double pp = 0.0;
  for (int k = 0; k < 12; ++k) pp += (double)p[k] * (double)p[k];
  o[0] = -s * s / (q.m * q.m * q.m);
  o[1] = s;
  o[2] = -(double)p[8];
  o[3] = 0.5 * pp;
}

// Reverse of qc_prox: given pb = dL/dp', add dL/dv to vb, dL/dx to xb (rows
// 6-11 and angles), dL/d(m, a_h, g_z, eps) to par.
template <typename T>
__device__ __forceinline__ void qc_prox_vjp(const QCNode<T>& n, const QCPar& q, T L,
                                            const T (&v)[12], const T (&pp)[12],
                                            const T (&pb)[12], T (&vb)[12], T (&xb)[12],
                                            double (&par)[4]) {
  const T al = T(1) + L * T(q.eps), ial = T(1) / al, irate = T(1) / (al + L);
  const T m = T(q.m), minv = T(1) / m;
  T alb = T(0);
  for (int k = 0; k < 6; ++k) {
    vb[k] += pb[k] * ial;
    xb[6 + k] += -L * ial * pb[k];
    alb += -pb[k] * pp[k] * ial;
  }
  for (int k = 9; k < 12; ++k) {
    vb[k] += pb[k] * irate;
    alb += -pb[k] * pp[k] * irate;               // d/d(al) of v/(al + L)
  }
  T w[3], b[3];
  for (int r = 0; r < 3; ++r) {
    w[r] = v[6 + r] - L * (T(q.ah) * n.a[r] - (r == 2 ? T(q.gz) : T(0)));
    b[r] = n.a[r] * minv;
  }
  const T bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  const T bw = b[0] * w[0] + b[1] * w[1] + b[2] * w[2];
  const T den = al + L * bb;
  const T f = L * bw / den;
  T wb[3], bbar[3], fb = T(0);
  for (int r = 0; r < 3; ++r) {
    wb[r] = pb[6 + r] * ial;
    fb += -pb[6 + r] * b[r] * ial;
    bbar[r] = -f * pb[6 + r] * ial;
    alb += -pb[6 + r] * pp[6 + r] * ial;
  }
  const T bwb = fb * L / den;
  const T denb = -fb * f / den;
  alb += denb;
  const T bbb = L * denb;
  for (int r = 0; r < 3; ++r) {
    bbar[r] += bwb * w[r] + T(2) * bbb * b[r];
    wb[r] += bwb * b[r];
  }
  T ab[3];
  double mb = 0.0, ahb = 0.0, gzb = 0.0;
  for (int r = 0; r < 3; ++r) {
    ab[r] = bbar[r] * minv;
    mb += -(double)(bbar[r] * n.a[r]) / ((double)q.m * q.m);
    vb[6 + r] += wb[r];
    ab[r] += -L * T(q.ah) * wb[r];
    ahb += -(double)(L * wb[r] * n.a[r]);
  }
  gzb += (double)(L * wb[2]);
  for (int c = 0; c < 3; ++c)
    xb[3 + c] += n.J[c] * ab[0] + n.J[3 + c] * ab[1] + n.J[6 + c] * ab[2];
  par[0] += mb;
  par[1] += ahb;
  par[2] += gzb;
  par[3] += (double)(L * alb);                    // al = 1 + L eps
}

// Reverse of qc_gradx: given gb = dL/dg, add dL/dx (angles) to xb, dL/dp to pb,
// dL/d(m, a_h) to par.
template <typename T>
__device__ __forceinline__ void qc_gradx_vjp(const QCNode<T>& n, const QCPar& q, const T (&p)[12],
                                             const T (&gb)[12], T (&xb)[12], T (&pb)[12],
                                             double (&par)[4]) {
  const T minv = T(1.0 / q.m);
  for (int k = 0; k < 3; ++k) { pb[k] += gb[6 + k]; pb[3 + k] += gb[9 + k]; }
  T qv[3] = {p[6], p[7], p[8]};
  const T s = n.a[0] * qv[0] + n.a[1] * qv[1] + n.a[2] * qv[2];
  const T coef = T(q.ah) + s * minv * minv;
  T h[3], hb[3], coefb = T(0);
  for (int c = 0; c < 3; ++c) {
    h[c] = n.J[c] * qv[0] + n.J[3 + c] * qv[1] + n.J[6 + c] * qv[2];
    coefb += gb[3 + c] * h[c];
    hb[c] = coef * gb[3 + c];
  }
  T qb[3], Jb[9];
  for (int r = 0; r < 3; ++r) {
    qb[r] = n.J[3 * r] * hb[0] + n.J[3 * r + 1] * hb[1] + n.J[3 * r + 2] * hb[2];
    for (int c = 0; c < 3; ++c) Jb[3 * r + c] = qv[r] * hb[c];
  }
  par[1] += (double)coefb;
  const T sb = coefb * minv * minv;
  par[0] += -2.0 * (double)(s * coefb) / ((double)q.m * q.m * q.m);
  T ab[3];
  for (int r = 0; r < 3; ++r) { ab[r] = sb * qv[r]; qb[r] += sb * n.a[r]; }
  for (int r = 0; r < 3; ++r) pb[6 + r] += qb[r];
  for (int k = 0; k < 3; ++k) {
    T acc = n.J[k] * ab[0] + n.J[3 + k] * ab[1] + n.J[6 + k] * ab[2];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) acc += Jb[3 * r + c] * n.H2[9 * r + 3 * c + k];
    xb[3 + k] += acc;
  }
}

template <typename T, int D, int G>
struct AdjShared {
  T zs[32 * G][D];
  T ps[32 * G][D];
  T node0[D];
  double red[G][2 * D + 4 + 1];
  unsigned long long item;
};

// FAM 0: quadratic (H = |p|^2 / 2), 1: quadcopter
template <typename T, int FAM, int D, int G>
__global__ void __launch_bounds__(32 * G) adjoint_kernel(const AdjArgs<T> a) {
  __shared__ AdjShared<T, D, G> sh;
  const int tid = threadIdx.x, lane = tid & 31, wg = tid >> 5;
  const int gl = tid, j = gl + 1;                 // this lane's node
  const int N = a.N;
  const bool mine = j <= N;
  const QCPar qp{a.qc_m, a.qc_ah, a.qc_gz, a.qc_eps};
  const T sig = a.sig, tau = a.tau, th = a.th;
  const size_t state = (size_t)3 * (N + 1) * D;   // one checkpoint
  T* work = a.work + (size_t)blockIdx.x * (size_t)(a.K_cap / a.C + 1) * state;

  for (;;) {
    __syncthreads();
    if (tid == 0) sh.item = atomicAdd(a.counter, 1ull);
    __syncthreads();
    const int64_t b = (int64_t)sh.item;
    if (b >= a.B) break;
    const int K = a.iters[b];
    if (K < 0 || K > a.K_cap) {
      if (tid == 0)
        for (int k = 0; k < D; ++k) a.dxq[b * D + k] = __longlong_as_double(0x7ff8000000000000ll);
      continue;
    }
    const double delta_d = a.t[b] / N;
    const T delta = T(a.t[b]) / T(N);
    const T L = sig * delta, taud = tau * delta;
    const uint64_t gid = (uint64_t)(a.point_offset + b);
    T ginv[D], goff[D];
    for (int k = 0; k < D; ++k) {
      ginv[k] = T(1.0 / (1.0 + (double)tau * a.W2[k]));
      goff[k] = T((double)tau * a.W2[k] * a.c[k]) * ginv[k];
    }

    // ---- state of this lane: node j (x, p, z); lane 0 also node 0 (x0, z0)
    T x[D], p[D], z[D], x0[D], z0[D];
    const InitGuess<T> ig(a.radius);                // the solver's initial guess
    auto init_state = [&]() {
      for (int k = 0; k < D; ++k) {
        const double xq = a.xq[b * D + k];
        x[k] = (j < N) ? ig.x(xq, a.seed, gid, j, k) : T(xq);
        p[k] = mine ? ig.p(a.seed, gid, j, k) : T(0);
        z[k] = x[k];
        x0[k] = ig.x(xq, a.seed, gid, 0, k);
        z0[k] = x0[k];
      }
    };
    // one forward iteration (the solver's step, one node per lane)
    auto step = [&]() {
      for (int k = 0; k < D; ++k) sh.zs[gl][k] = z[k];
      __syncthreads();
      T zl[D];
      for (int k = 0; k < D; ++k) zl[k] = (gl > 0) ? sh.zs[gl - 1][k] : z0[k];
      T pn[D];
      QCNode<T> nd;
      if (mine) {
        T v[D];
        for (int k = 0; k < D; ++k) v[k] = p[k] + sig * (z[k] - zl[k]);
        if constexpr (FAM == 1) {
          qc_node<T>(reinterpret_cast<const T(&)[12]>(x), nd);
          qc_prox<T>(nd, qp, L, reinterpret_cast<const T(&)[12]>(x), reinterpret_cast<const T(&)[12]>(v),
                     reinterpret_cast<T(&)[12]>(pn));
        } else {
          for (int k = 0; k < D; ++k) pn[k] = v[k] / (T(1) + L);
        }
      } else {
        for (int k = 0; k < D; ++k) pn[k] = T(0);
      }
      for (int k = 0; k < D; ++k) sh.ps[gl][k] = pn[k];
      __syncthreads();
      if (gl == 0) {
        for (int k = 0; k < D; ++k) {
          const T xn = (x0[k] + tau * pn[k]) * ginv[k] + goff[k];
          z0[k] = xn + th * (xn - x0[k]);
          x0[k] = xn;
        }
      }
      if (mine && j < N) {
        T g[D];
        if constexpr (FAM == 1)
          qc_gradx<T>(nd, qp, reinterpret_cast<const T(&)[12]>(pn), reinterpret_cast<T(&)[12]>(g));
        else
          for (int k = 0; k < D; ++k) g[k] = T(0);
        for (int k = 0; k < D; ++k) {
          const T xn = x[k] - tau * (pn[k] - sh.ps[gl + 1][k]) + taud * g[k];
          z[k] = xn + th * (xn - x[k]);
          x[k] = xn;
        }
      }
      for (int k = 0; k < D; ++k) p[k] = pn[k];
      __syncthreads();
    };
    auto save = [&](int slot) {
      T* s = work + (size_t)slot * state;
      if (mine)
        for (int k = 0; k < D; ++k) {
          s[(size_t)j * D + k] = x[k];
          s[(size_t)(N + 1) * D + (size_t)j * D + k] = p[k];
          s[(size_t)2 * (N + 1) * D + (size_t)j * D + k] = z[k];
        }
      if (gl == 0)
        for (int k = 0; k < D; ++k) {
          s[k] = x0[k];
          s[(size_t)2 * (N + 1) * D + k] = z0[k];
        }
    };
    auto load = [&](int slot) {
      const T* s = work + (size_t)slot * state;
      __syncthreads();
      if (mine)
        for (int k = 0; k < D; ++k) {
          x[k] = s[(size_t)j * D + k];
          p[k] = s[(size_t)(N + 1) * D + (size_t)j * D + k];
          z[k] = s[(size_t)2 * (N + 1) * D + (size_t)j * D + k];
        }
      if (gl == 0)
        for (int k = 0; k < D; ++k) {
          x0[k] = s[k];
          z0[k] = s[(size_t)2 * (N + 1) * D + k];
        }
      __syncthreads();
    };

    // ---- forward with checkpoints
    init_state();
    for (int k = 0; k < K; ++k) {
      if (k % a.C == 0) save(k / a.C);
      step();
    }
    __syncthreads();

    // ---- adjoint of the value at s^K
    double parb[4] = {0, 0, 0, 0};
    double Wb[D], cb[D];
    for (int k = 0; k < D; ++k) { Wb[k] = 0.0; cb[k] = 0.0; }
    T xb[D], pb[D], zb[D], x0b[D], z0b[D];
    {
      for (int k = 0; k < D; ++k) { sh.ps[gl][k] = p[k]; sh.zs[gl][k] = x[k]; }
      __syncthreads();
      T gx[D], gp[D];
      QCNode<T> nd;
      if (mine) {
        if constexpr (FAM == 1) {
          qc_node<T>(reinterpret_cast<const T(&)[12]>(x), nd);
          qc_gradx<T>(nd, qp, reinterpret_cast<const T(&)[12]>(p), reinterpret_cast<T(&)[12]>(gx));
          qc_gradp<T>(nd, qp, reinterpret_cast<const T(&)[12]>(x), reinterpret_cast<const T(&)[12]>(p),
                      reinterpret_cast<T(&)[12]>(gp));
          double hp[4];
          qc_dHdpar<T>(nd, qp, reinterpret_cast<const T(&)[12]>(p), hp);
          for (int i = 0; i < 4; ++i) parb[i] += -delta_d * hp[i];
        } else {
          for (int k = 0; k < D; ++k) { gx[k] = T(0); gp[k] = p[k]; }
        }
      }
      for (int k = 0; k < D; ++k) {
        const T pr = (mine && j < N) ? sh.ps[gl + 1][k] : T(0);
        const T xl = (gl > 0) ? sh.zs[gl - 1][k] : x0[k];
        xb[k] = mine ? (p[k] - pr - delta * gx[k]) : T(0);     // node N: p_N - delta grad_x H
        pb[k] = mine ? (x[k] - xl - delta * gp[k]) : T(0);
        zb[k] = T(0);
        x0b[k] = T(0); z0b[k] = T(0);
      }
      if (gl == 0)
        for (int k = 0; k < D; ++k) {
          const double e = (double)x0[k] - a.c[k];
          x0b[k] = T(a.W2[k] * e) - p[k];                          // grad g(x_0) - p_1
          Wb[k] += a.W[k] * e * e;
          cb[k] += -a.W2[k] * e;
        }
      __syncthreads();
    }

    // ---- backward sweep, newest segment first
    const int nseg = (K + a.C - 1) / a.C;
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
      const int k0 = sgi * a.C;
      const int k1 = min(K, k0 + a.C);
      for (int k = k1 - 1; k >= k0; --k) {
        load(sgi);
        for (int r = k0; r < k; ++r) step();        // s^k
        // intermediates of step k at s^k
        for (int kk = 0; kk < D; ++kk) sh.zs[gl][kk] = z[kk];
        __syncthreads();
        T zl[D], v[D], pn[D];
        for (int kk = 0; kk < D; ++kk) zl[kk] = (gl > 0) ? sh.zs[gl - 1][kk] : z0[kk];
        QCNode<T> nd;
        if (mine) {
          for (int kk = 0; kk < D; ++kk) v[kk] = p[kk] + sig * (z[kk] - zl[kk]);
          if constexpr (FAM == 1) {
            qc_node<T>(reinterpret_cast<const T(&)[12]>(x), nd);
            qc_prox<T>(nd, qp, L, reinterpret_cast<const T(&)[12]>(x),
                       reinterpret_cast<const T(&)[12]>(v), reinterpret_cast<T(&)[12]>(pn));
          } else {
            for (int kk = 0; kk < D; ++kk) pn[kk] = v[kk] / (T(1) + L);
          }
        } else {
          for (int kk = 0; kk < D; ++kk) { v[kk] = T(0); pn[kk] = T(0); }
        }
        __syncthreads();
        // (xb, pb, zb) are the adjoints of s^{k+1}; build those of s^k
        T nxb[D], npb[D], nzb[D], pnb[D];
        for (int kk = 0; kk < D; ++kk) { nxb[kk] = T(0); npb[kk] = T(0); nzb[kk] = T(0); pnb[kk] = pb[kk]; }
        T xpb[D];                                     // adjoint of x^{k+1}_j after z' = x' + th (x' - x)
        if (mine && j < N) {
          for (int kk = 0; kk < D; ++kk) {
            xpb[kk] = xb[kk] + (T(1) + th) * zb[kk];
            nxb[kk] += -th * zb[kk] + xpb[kk];
            pnb[kk] += -tau * xpb[kk];
          }
          T gb[D];
          for (int kk = 0; kk < D; ++kk) gb[kk] = taud * xpb[kk];
          if constexpr (FAM == 1)
            qc_gradx_vjp<T>(nd, qp, reinterpret_cast<const T(&)[12]>(pn), reinterpret_cast<const T(&)[12]>(gb),
                            reinterpret_cast<T(&)[12]>(nxb), reinterpret_cast<T(&)[12]>(pnb), parb);
        } else {
          for (int kk = 0; kk < D; ++kk) xpb[kk] = T(0);
          if (mine)                                   // node N: x' = x, z' = x
            for (int kk = 0; kk < D; ++kk) nxb[kk] += xb[kk] + zb[kk];
        }
        // p'_{j} also enters x'_{j-1} (+tau) and, for j = 1, x'_0
        for (int kk = 0; kk < D; ++kk) sh.ps[gl][kk] = tau * xpb[kk];
        __syncthreads();
        if (mine && gl > 0)
          for (int kk = 0; kk < D; ++kk) pnb[kk] += sh.ps[gl - 1][kk];
        if (gl == 0) {
          for (int kk = 0; kk < D; ++kk) {
            // x0' = (x0 + tau p'_1) ginv + goff; z0' = x0' + th (x0' - x0)
            const T x0p = (x0[kk] + tau * pn[kk]) * ginv[kk] + goff[kk];
            const T x0pb = x0b[kk] + (T(1) + th) * z0b[kk];
            const T nx0b = -th * z0b[kk] + x0pb * ginv[kk];
            pnb[kk] += x0pb * ginv[kk] * tau;
            const double w2 = a.W2[kk];
            Wb[kk] += (double)x0pb * 2.0 * (double)tau * a.W[kk] * (a.c[kk] - (double)x0p) *
                      (double)ginv[kk];
            cb[kk] += (double)x0pb * (double)tau * w2 * (double)ginv[kk];
            x0b[kk] = nx0b;
            z0b[kk] = T(0);
          }
        }
        // dual step: p'_j = prox(x_j, v_j), v_j = p_j + sig (z_j - z_{j-1})
        T vb[D];
        for (int kk = 0; kk < D; ++kk) vb[kk] = T(0);
        if (mine) {
          if constexpr (FAM == 1)
            qc_prox_vjp<T>(nd, qp, L, reinterpret_cast<const T(&)[12]>(v), reinterpret_cast<const T(&)[12]>(pn),
                           reinterpret_cast<const T(&)[12]>(pnb), reinterpret_cast<T(&)[12]>(vb),
                           reinterpret_cast<T(&)[12]>(nxb), parb);
          else
            for (int kk = 0; kk < D; ++kk) vb[kk] = pnb[kk] / (T(1) + L);
          for (int kk = 0; kk < D; ++kk) { npb[kk] += vb[kk]; nzb[kk] += sig * vb[kk]; }
        }
        __syncthreads();
        for (int kk = 0; kk < D; ++kk) sh.zs[gl][kk] = -sig * vb[kk];
        __syncthreads();
        if (mine && j < N)
          for (int kk = 0; kk < D; ++kk) nzb[kk] += sh.zs[gl + 1][kk];
        if (gl == 0)
          for (int kk = 0; kk < D; ++kk) z0b[kk] += sh.zs[0][kk];
        for (int kk = 0; kk < D; ++kk) { xb[kk] = nxb[kk]; pb[kk] = npb[kk]; zb[kk] = nzb[kk]; }
        __syncthreads();
      }
    }

    // ---- s^0 depends on x through x^0_j = x + r u (j < N), x^0_N = x, z^0 = x^0
    double xqb[D];
    for (int k = 0; k < D; ++k) xqb[k] = mine ? (double)xb[k] + (double)zb[k] : 0.0;
    if (gl == 0)
      for (int k = 0; k < D; ++k) xqb[k] += (double)x0b[k] + (double)z0b[k];
    const double wb = a.w[b];
    for (int k = 0; k < D; ++k) xqb[k] = warp_sum<double>(xqb[k]);
    for (int i = 0; i < 4; ++i) parb[i] = warp_sum<double>(parb[i]);
    if (lane == 0) {
      for (int k = 0; k < D; ++k) sh.red[wg][k] = xqb[k];
      for (int i = 0; i < 4; ++i) sh.red[wg][2 * D + i] = parb[i];
    }
    __syncthreads();
    if (tid == 0) {
      for (int k = 0; k < D; ++k) {
        double s = 0.0;
        for (int w = 0; w < G; ++w) s += sh.red[w][k];
        a.dxq[b * D + k] = wb * s;
        atomicAdd(&a.dW[k], wb * Wb[k]);
        atomicAdd(&a.dc[k], wb * cb[k]);
      }
      if (FAM == 1)
        for (int i = 0; i < 4; ++i) {
          double s = 0.0;
          for (int w = 0; w < G; ++w) s += sh.red[w][2 * D + i];
          atomicAdd(&a.ddyn[i], wb * s);
        }
    }
  }
}

template <typename T, int FAM, int D>
hj_status launch_adj(const AdjArgs<T>& a, int grid, cudaStream_t s) {
  const int G = (a.N + 31) / 32;
  switch (G) {
    case 1: adjoint_kernel<T, FAM, D, 1><<<grid, 32, 0, s>>>(a); break;
    case 2: adjoint_kernel<T, FAM, D, 2><<<grid, 64, 0, s>>>(a); break;
    case 3: case 4: adjoint_kernel<T, FAM, D, 4><<<grid, 128, 0, s>>>(a); break;
    case 5: case 6: case 7: case 8:
      // FP64 12-D slots for 256 lanes exceed the 48 KB of static shared memory
      if constexpr (sizeof(AdjShared<T, D, 8>) > 48 * 1024) return HJ_ERR_UNSUPPORTED;
      else adjoint_kernel<T, FAM, D, 8><<<grid, 256, 0, s>>>(a);
      break;
    default: return HJ_ERR_UNSUPPORTED;
  }
  return cudaGetLastError() == cudaSuccess ? HJ_OK : HJ_ERR_CUDA;
}

}  // namespace

// Grid used by the adjoint (its workspace is per CTA).
int adjoint_grid(int64_t B) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t g = (int64_t)nsm * 4;
  return (int)(B < g ? (B > 0 ? B : 1) : g);
}

template <typename T>
hj_status launch_adjoint(int family, const AdjArgs<T>& a, int grid, cudaStream_t s) {
  if (a.N < 1 || a.N > 256) return HJ_ERR_UNSUPPORTED;
  if (family == HJ_FAMILY_QUADCOPTER && a.d == 12) return launch_adj<T, 1, 12>(a, grid, s);
  if (family == HJ_FAMILY_QUADRATIC) {
    switch (a.d) {
      case 1: return launch_adj<T, 0, 1>(a, grid, s);
      case 2: return launch_adj<T, 0, 2>(a, grid, s);
      case 3: return launch_adj<T, 0, 3>(a, grid, s);
      case 4: return launch_adj<T, 0, 4>(a, grid, s);
      default: return HJ_ERR_UNSUPPORTED;
    }
  }
  return HJ_ERR_UNSUPPORTED;
}

template hj_status launch_adjoint<float>(int, const AdjArgs<float>&, int, cudaStream_t);
template hj_status launch_adjoint<double>(int, const AdjArgs<double>&, int, cudaStream_t);

}  // namespace hj
