// Per-node Hamiltonian kernels for the register-resident solver.
//
// Each family provides, for one time node j with state x_j (D values):
//   context(x, ctx)         quantities of H at x_j^k shared by the dual prox and
//                           the x-gradient (H is evaluated once per node and
//                           iteration, at x^k as in Appendix Algorithm A.1)
//   point(lam)              per-point constants of the prox (lam = sigma delta)
//   prox(ctx, pc, x, v)     v <- argmin_p lam*H(x, p) + |p - v|^2/2
//   gradx(ctx, x, p, g)     g <- grad_x H(x, p)
//   H64(x, p)               H in double from the iterates, for the value
//                           (fval of Algorithm 1); converts element by element
//   Ht(x, p)                H in the iterate type (the FP32 path's value terms)
//   prox_first(ctx, pc, x, v, hs, hc)
//                           the Hopf form's node-1 dual step: the prox of
//                           sigma g* + lam H, hs = sigma / W^2, hc = sigma c
//   prox_mix(cr, cl, pc, wr, wl, xr, xl, v)
//                           v <- argmin_p lam (wr H(xr, p) + wl H(xl, p)) + |p - v|^2/2
//                           for weights wr + wl = 1 (forward-Euler and trapezoid
//                           schemes; cr, cl the contexts at xr, xl)
//   kkt_node(x, xl, p, pr, delta, s, r3)
//                           node j's part of the residual of the discrete
//                           characteristic equations (Section 4), in FP64 from
//                           the iterates x = x_j, xl = x_{j-1}, p = p_j, pr = p_{j+1}:
//                           max_k |x_j - x_{j-1} - delta grad_p H(x_j, p_j)|_k and,
//                           with r3, max_k |p_{j+1} - p_j + delta grad_x H(x_j, p_j)|_k
// All families have L = |u|^2/2, so H = <p, f0(x)> + |B(x)^T p|^2/2 (Section 2).
#pragma once
#include <type_traits>

#include "hj_internal.cuh"

namespace hj {

template <typename T>
__device__ __forceinline__ void sin_cos(T x, T* s, T* c);
template <>
__device__ __forceinline__ void sin_cos<float>(float x, float* s, float* c) {
  __sincosf(x, s, c);
}
template <>
__device__ __forceinline__ void sin_cos<double>(double x, double* s, double* c) {
  sincos(x, s, c);
}

// Elementwise operations on coordinate arrays.  FP32 issues the packed
// two-wide instructions (one instruction per pair of coordinates, each element
// rounded once exactly as the scalar operation); FP64 and odd tails are scalar.
template <typename T, int D>
__device__ __forceinline__ void v_sub(T (&r)[D], const T (&a)[D], const T (&b)[D]) {
  int k0 = 0;
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int k = 0; k + 1 < D; k += 2) {
      const float2 o = __fadd2_rn(make_float2(a[k], a[k + 1]), make_float2(-b[k], -b[k + 1]));
      r[k] = o.x; r[k + 1] = o.y;
    }
    k0 = D - D % 2;
  }
#pragma unroll
  for (int k = k0; k < D; ++k) r[k] = a[k] - b[k];
}

// r = s * x + y
template <typename T, int D>
__device__ __forceinline__ void v_fma(T (&r)[D], T s, const T (&x)[D], const T (&y)[D]) {
  int k0 = 0;
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int k = 0; k + 1 < D; k += 2) {
      const float2 o = __ffma2_rn(make_float2(s, s), make_float2(x[k], x[k + 1]),
                                  make_float2(y[k], y[k + 1]));
      r[k] = o.x; r[k + 1] = o.y;
    }
    k0 = D - D % 2;
  }
#pragma unroll
  for (int k = k0; k < D; ++k) r[k] = fma(s, x[k], y[k]);
}

// r = s * x - y
template <typename T, int D>
__device__ __forceinline__ void v_fms(T (&r)[D], T s, const T (&x)[D], const T (&y)[D]) {
  int k0 = 0;
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int k = 0; k + 1 < D; k += 2) {
      const float2 o = __ffma2_rn(make_float2(s, s), make_float2(x[k], x[k + 1]),
                                  make_float2(-y[k], -y[k + 1]));
      r[k] = o.x; r[k + 1] = o.y;
    }
    k0 = D - D % 2;
  }
#pragma unroll
  for (int k = k0; k < D; ++k) r[k] = fma(s, x[k], -y[k]);
}

// acc += sum_k e_k^2 (pairs accumulated two-wide, folded at the end)
template <typename T, int D>
__device__ __forceinline__ T v_sumsq(const T (&e)[D]) {
  T acc = T(0);
  int k0 = 0;
  if constexpr (sizeof(T) == 4) {
    float2 a2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k + 1 < D; k += 2) {
      const float2 v = make_float2(e[k], e[k + 1]);
      a2 = __ffma2_rn(v, v, a2);
    }
    acc = a2.x + a2.y;
    k0 = D - D % 2;
  }
#pragma unroll
  for (int k = k0; k < D; ++k) acc = fma(e[k], e[k], acc);
  return acc;
}

// a / b; FP32 uses the fast reciprocal-based division (2 ulp).
template <typename T>
__device__ __forceinline__ T fdiv(T a, T b) { return a / b; }
template <>
__device__ __forceinline__ float fdiv<float>(float a, float b) { return __fdividef(a, b); }

template <typename T>
__device__ __forceinline__ T tanh_t(T y) { return tanh(y); }
template <>
__device__ __forceinline__ float tanh_t<float>(float y) { return tanhf(y); }

template <typename T>
__device__ __forceinline__ T exp_t(T y) { return exp(y); }
template <>
__device__ __forceinline__ float exp_t<float>(float y) { return __expf(y); }

template <typename T>
__device__ __forceinline__ T sqrt_t(T y) { return sqrt(y); }
template <>
__device__ __forceinline__ float sqrt_t<float>(float y) { return sqrtf(y); }


// ---------------------------------------------------------------- H = |p|^2/2
template <typename T, int D>
struct FamQuadratic {
  static constexpr bool kHasGradX = false;
  static constexpr bool kGame = false;
  static constexpr bool kTimeDep = false;
  struct Shared {};
  struct Ctx {};
  struct PC { T s, lam; };
  __device__ static void load_shared(const SolveArgs<T>&, Shared&) {}
  __device__ FamQuadratic(const SolveArgs<T>&, const Shared&) {}
  __device__ __forceinline__ PC point(T lam) const { return PC{T(1) / (T(1) + lam), lam}; }
  __device__ __forceinline__ void context(const T (&)[D], Ctx&) const {}
  __device__ __forceinline__ void prox(const Ctx&, const PC& pc, const T (&)[D], T (&v)[D]) const {
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] *= pc.s;
  }
  // Hopf form, node 1: argmin_p sigma g*(p) + lam H + |p - v|^2/2 with
  // g*(p) = <p, c> + 1/2 sum p_k^2 / W_k^2; hs = sigma / W^2, hc = sigma c.
  __device__ __forceinline__ void prox_first(const Ctx&, const PC& pc, const T (&)[D], T (&v)[D],
                                             const T* hs, const T* hc) const {
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = fdiv<T>(v[k] - hc[k], T(1) + pc.lam + hs[k]);
  }
  __device__ __forceinline__ void gradx(const Ctx&, const T (&)[D], const T (&)[D], T (&g)[D]) const {
#pragma unroll
    for (int k = 0; k < D; ++k) g[k] = T(0);
  }
  __device__ __forceinline__ double H64(const T (&)[D], const T (&p)[D]) const {
    double h = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) h += (double)p[k] * (double)p[k];
    return 0.5 * h;
  }
  __device__ __forceinline__ T Ht(const T (&)[D], const T (&p)[D]) const {
    T h = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) h += p[k] * p[k];
    return T(0.5) * h;
  }
  // grad_p H = p, grad_x H = 0
  __device__ double kkt_node(const T (&x)[D], const T (&xl)[D], const T (&p)[D], const T (&pr)[D],
                             double delta, double, bool r3) const {
    double r = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double pk = (double)p[k];
      r = max_nan(r, fabs((double)x[k] - (double)xl[k] - delta * pk));
      if (r3) r = max_nan(r, fabs((double)pr[k] - pk));
    }
    return r;
  }
};

// ---------------------------------------------------------------- quadcopter, D = 12
// State (x, y, z, psi, theta, phi, then rates).  Thrust direction
//   a = (s_phi s_psi + c_phi c_psi s_theta, -c_psi s_phi + c_phi s_theta s_psi, c_theta c_phi)
// f0 = (v_pos, v_ang, a_h a - g_z e3, 0), B = [(0_6; a/m; 0_3) | e10 | e11 | e12],
// H = <p, f0> + |B^T p|^2/2 + eps |p|^2/2.
template <typename T, int D>
struct FamQuadcopter {
  static_assert(D == 12, "quadcopter state is 12-D");
  static constexpr bool kHasGradX = true;
  static constexpr bool kKktInIterType = true;   // kkt_node: FP32 iterates in FP32
  static constexpr bool kGame = false;
  static constexpr bool kTimeDep = false;
  struct Shared {};
  struct Ctx { T a[3]; T J[9]; };
  T m_inv, ah, gz, eps;
  double m64, ah64, gz64, eps64;
  __device__ static void load_shared(const SolveArgs<T>&, Shared&) {}
  __device__ FamQuadcopter(const SolveArgs<T>& s, const Shared&)
      : m_inv(s.qc_t[0]), ah(s.qc_t[1]), gz(s.qc_t[2]), eps(s.qc_t[3]),
        m64(s.qc_m), ah64(s.qc_ah), gz64(s.qc_gz), eps64(s.qc_eps) {}

  template <typename U>
  __device__ __forceinline__ static void thrust(const U psi, const U th, const U ph, U (&a)[3],
                                                U (&J)[9]) {
    U sps, cps, sth, cth, sph, cph;
    sin_cos<U>(psi, &sps, &cps);
    sin_cos<U>(th, &sth, &cth);
    sin_cos<U>(ph, &sph, &cph);
    const U cc = cph * cps, cs = cph * sps, sc = sph * cps, ss = sph * sps;
    a[0] = ss + cc * sth;
    a[1] = -sc + cs * sth;
    a[2] = cth * cph;
    // J[3*r + k] = d a_r / d (psi, theta, phi)_k
    J[0] = sc - cs * sth;
    J[1] = cc * cth;
    J[2] = cs - sc * sth;
    J[3] = ss + cc * sth;
    J[4] = cs * cth;
    J[5] = -cc - ss * sth;
    J[6] = U(0);
    J[7] = -sth * cph;
    J[8] = -cth * sph;
  }

  __device__ __forceinline__ void context(const T (&x)[D], Ctx& c) const {
    thrust<T>(x[3], x[4], x[5], c.a, c.J);
  }

  // Per-point constants of the prox: al = 1 + lam eps and the reciprocals used below.
  struct PC { T lam, ial, irate, lam_ah, lam_gz, al; };
  __device__ __forceinline__ PC point(T lam) const {
    PC c;
    c.lam = lam;
    c.al = T(1) + lam * eps;
    c.ial = T(1) / c.al;
    c.irate = T(1) / (c.al + lam);
    c.lam_ah = lam * ah;
    c.lam_gz = lam * gz;
    return c;
  }

  // ((1 + lam eps) I + lam B B^T) p = v - lam f0.  Rows 0-5 and 9-11 decouple;
  // rows 6-8 are a rank-1 update of a scaled identity (Sherman-Morrison).
  __device__ __forceinline__ void prox(const Ctx& c, const PC& pc, const T (&x)[D],
                                       T (&v)[D]) const {
    const T lam = pc.lam, ial = pc.ial;
    if constexpr (sizeof(T) == 4) {
      // rows 0-5: (v - lam x_{6..11}) * ial, rows 9-10 scaled, two-wide
#pragma unroll
      for (int k = 0; k < 6; k += 2) {
        const float2 t = __ffma2_rn(make_float2(-lam, -lam), make_float2(x[6 + k], x[7 + k]),
                                    make_float2(v[k], v[k + 1]));
        const float2 o = __fmul2_rn(t, make_float2(ial, ial));
        v[k] = o.x; v[k + 1] = o.y;
      }
      const float2 r = __fmul2_rn(make_float2(v[9], v[10]), make_float2(pc.irate, pc.irate));
      v[9] = r.x; v[10] = r.y;
      v[11] *= pc.irate;
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) v[k] = (v[k] - lam * x[6 + k]) * ial;
#pragma unroll
      for (int k = 0; k < 3; ++k) v[3 + k] = (v[3 + k] - lam * x[9 + k]) * ial;
#pragma unroll
      for (int k = 0; k < 3; ++k) v[9 + k] *= pc.irate;
    }
    const T w0 = v[6] - pc.lam_ah * c.a[0];
    const T w1 = v[7] - pc.lam_ah * c.a[1];
    const T w2 = v[8] - (pc.lam_ah * c.a[2] - pc.lam_gz);
    const T b0 = c.a[0] * m_inv, b1 = c.a[1] * m_inv, b2 = c.a[2] * m_inv;
    const T bb = b0 * b0 + b1 * b1 + b2 * b2;
    const T bw = b0 * w0 + b1 * w1 + b2 * w2;
    const T f = fdiv<T>(lam * bw, pc.al + lam * bb);
    v[6] = (w0 - f * b0) * ial;
    v[7] = (w1 - f * b1) * ial;
    v[8] = (w2 - f * b2) * ial;
  }

  // Mixed schemes: (al I + lam (wr B_r B_r^T + wl B_l B_l^T)) p = v - lam (wr f0(xr) + wl f0(xl)),
  // al = 1 + lam eps (wr + wl = 1).  Rows 0-5 and 9-11 decouple as above; rows
  // 6-8 carry two rank-1 terms, u = a_r/m and s = a_l/m with alpha = lam wr and
  // beta = lam wl.  With y = (w - alpha U u - beta S s) / al, U = u.y and S = s.y
  // solve the 2x2 system
  //   [al + alpha u.u, beta u.s; alpha u.s, al + beta s.s] [U; S] = [u.w; s.w].
  __device__ __forceinline__ void prox_mix(const Ctx& cr, const Ctx& cl, const PC& pc, T wr, T wl,
                                           const T (&xr)[D], const T (&xl)[D], T (&v)[D]) const {
    const T lam = pc.lam, ial = pc.ial;
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = (v[k] - lam * (wr * xr[6 + k] + wl * xl[6 + k])) * ial;
#pragma unroll
    for (int k = 9; k < 12; ++k) v[k] *= pc.irate;
    T w[3], u[3], sv[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      w[r] = v[6 + r] - (pc.lam_ah * (wr * cr.a[r] + wl * cl.a[r]) - (r == 2 ? pc.lam_gz : T(0)));
      u[r] = cr.a[r] * m_inv;
      sv[r] = cl.a[r] * m_inv;
    }
    const T al = pc.al, alpha = lam * wr, beta = lam * wl;
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const T ss = sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2];
    const T us = u[0] * sv[0] + u[1] * sv[1] + u[2] * sv[2];
    const T uw = u[0] * w[0] + u[1] * w[1] + u[2] * w[2];
    const T sw = sv[0] * w[0] + sv[1] * w[1] + sv[2] * w[2];
    const T m11 = al + alpha * uu, m22 = al + beta * ss;
    const T idet = fdiv<T>(T(1), m11 * m22 - alpha * beta * us * us);
    const T U = (m22 * uw - beta * us * sw) * idet;
    const T S = (m11 * sw - alpha * us * uw) * idet;
#pragma unroll
    for (int r = 0; r < 3; ++r) v[6 + r] = (w[r] - alpha * U * u[r] - beta * S * sv[r]) * ial;
  }

  // Hopf form, node 1: the prox above with sigma g*(p) added, g*(p) = <p, c> +
  // 1/2 sum p_k^2 / W_k^2 (hs = sigma / W^2, hc = sigma c):
  //   (diag(1 + lam eps + hs) + lam B B^T) p = v - hc - lam f0.
  // Rows 6-8 are a rank-1 update of the diagonal L = diag(1 + lam eps + hs_6..8):
  //   p = L^-1 w - L^-1 b (lam b^T L^-1 w) / (1 + lam b^T L^-1 b).
  __device__ __forceinline__ void prox_first(const Ctx& c, const PC& pc, const T (&x)[D],
                                             T (&v)[D], const T* hs, const T* hc) const {
    const T lam = pc.lam;
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = fdiv<T>(v[k] - hc[k] - lam * x[6 + k], pc.al + hs[k]);
#pragma unroll
    for (int k = 9; k < 12; ++k) v[k] = fdiv<T>(v[k] - hc[k], pc.al + lam + hs[k]);
    T y[3], q[3], b[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const T il = fdiv<T>(T(1), pc.al + hs[6 + r]);
      const T w = v[6 + r] - hc[6 + r] - (pc.lam_ah * c.a[r] - (r == 2 ? pc.lam_gz : T(0)));
      b[r] = c.a[r] * m_inv;
      y[r] = il * w;
      q[r] = il * b[r];
    }
    const T by = b[0] * y[0] + b[1] * y[1] + b[2] * y[2];
    const T bq = b[0] * q[0] + b[1] * q[1] + b[2] * q[2];
    const T f = fdiv<T>(lam * by, T(1) + lam * bq);
#pragma unroll
    for (int r = 0; r < 3; ++r) v[6 + r] = y[r] - f * q[r];
  }

  // The Hopf form with one code path for every lane: each row k of the prox
  // takes an offset off_k and a reciprocal diagonal dinv_k from a per-lane table,
  //   rows 0-5:  p_k = (v_k - off_k - lam x_{6+k}) dinv_k,
  //   rows 9-11: p_k = (v_k - off_k) dinv_k,
  //   rows 6-8:  L^-1 = diag(dinv_6..8), w = v - off - lam (a_h a - g_z e3),
  //              p = L^-1 w - L^-1 b (lam b^T L^-1 w) / (1 + lam b^T L^-1 b), b = a / m,
  // which is prox (off = 0, dinv = 1 / al, 1 / (al + lam) on rows 9-11) for a
  // plain node and prox_first (off = hc, dinv = 1 / (al + hs), 1 / (al + lam + hs)
  // on rows 9-11) for node 1, so the lane of node 1 no longer runs its own code.
  static constexpr bool kHopfTable = true;
  __device__ __forceinline__ void hopf_row(const PC& pc, const T* hs, const T* hc, int k,
                                           T& off_plain, T& dinv_plain, T& off_first,
                                           T& dinv_first) const {
    const bool torque = k >= 9;
    off_plain = T(0);
    dinv_plain = torque ? pc.irate : pc.ial;
    off_first = hc[k];
    dinv_first = T(1) / (pc.al + (torque ? pc.lam : T(0)) + hs[k]);
  }
  __device__ __forceinline__ void prox_hopf(const Ctx& c, const PC& pc, const T (&x)[D], T (&v)[D],
                                            const T* off, const T* dinv) const {
    const T lam = pc.lam;
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = (v[k] - off[k] - lam * x[6 + k]) * dinv[k];
#pragma unroll
    for (int k = 9; k < 12; ++k) v[k] = (v[k] - off[k]) * dinv[k];
    T y[3], q[3], b[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const T w = v[6 + r] - off[6 + r] - (pc.lam_ah * c.a[r] - (r == 2 ? pc.lam_gz : T(0)));
      b[r] = c.a[r] * m_inv;
      y[r] = dinv[6 + r] * w;
      q[r] = dinv[6 + r] * b[r];
    }
    const T by = b[0] * y[0] + b[1] * y[1] + b[2] * y[2];
    const T bq = b[0] * q[0] + b[1] * q[1] + b[2] * q[2];
    const T f = fdiv<T>(lam * by, T(1) + lam * bq);
#pragma unroll
    for (int r = 0; r < 3; ++r) v[6 + r] = y[r] - f * q[r];
  }

  __device__ __forceinline__ void gradx(const Ctx& c, const T (&)[D], const T (&p)[D],
                                        T (&g)[D]) const {
    const T u0 = (c.a[0] * p[6] + c.a[1] * p[7] + c.a[2] * p[8]) * m_inv;
    const T coef = ah + u0 * m_inv;
    g[0] = g[1] = g[2] = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      g[3 + k] = coef * (c.J[k] * p[6] + c.J[3 + k] * p[7] + c.J[6 + k] * p[8]);
#pragma unroll
    for (int k = 0; k < 3; ++k) g[6 + k] = p[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) g[9 + k] = p[3 + k];
  }

  __device__ __forceinline__ double H64(const T (&x)[D], const T (&p)[D]) const {
    double a[3], J[9];
    thrust<double>((double)x[3], (double)x[4], (double)x[5], a, J);
    double h = 0.0, pp = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      h += (double)p[k] * (double)x[6 + k] + (double)p[3 + k] * (double)x[9 + k];
    const double s = a[0] * (double)p[6] + a[1] * (double)p[7] + a[2] * (double)p[8];
    h += ah64 * s - gz64 * (double)p[8];
    const double u0 = s / m64;
#pragma unroll
    for (int k = 0; k < D; ++k) pp += (double)p[k] * (double)p[k];
    double rr = 0.0;
#pragma unroll
    for (int k = 9; k < 12; ++k) rr += (double)p[k] * (double)p[k];
    return h + 0.5 * (u0 * u0 + rr) + 0.5 * eps64 * pp;
  }
  __device__ __forceinline__ T Ht(const T (&x)[D], const T (&p)[D]) const {
    T a[3], J[9];
    thrust<T>(x[3], x[4], x[5], a, J);
    T h = T(0), pp = T(0), rr = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) h += p[k] * x[6 + k] + p[3 + k] * x[9 + k];
    const T s = a[0] * p[6] + a[1] * p[7] + a[2] * p[8];
    h += ah * s - gz * p[8];
    const T u0 = s * m_inv;
#pragma unroll
    for (int k = 0; k < D; ++k) pp += p[k] * p[k];
#pragma unroll
    for (int k = 9; k < 12; ++k) rr += p[k] * p[k];
    return h + T(0.5) * (u0 * u0 + rr) + T(0.5) * eps * pp;
  }
  // grad_p H = f0 + B B^T p + eps p: (v_pos, v_ang, a_h a - g_z e3 + a u0 / m, tau) + eps p
  // with u0 = <a, p_7..9> / m; grad_x H = (0, (a_h + u0 / m) J^T p_7..9, p_1..3, p_4..6).
  // Evaluated in the iterate type: FP64 iterates in FP64 throughout; FP32 iterates
  // in FP32 with the sines and cosines from the accurate sincosf (2 ulp), which
  // keeps the residual's evaluation error below about 16 units of 2^-24 times the
  // magnitudes that enter it (|x_j - x_{j-1}|, |p_{j+1} - p_j| and delta times the
  // terms of grad H), that is below the rounding of the FP32 iterates themselves
  // (FP64 arithmetic here runs at 1/64 of the FP32 rate and would cost the solve
  // several per cent).
  template <typename E>
  __device__ __forceinline__ static E max_keep_nan(E a, E b) { return (a > b || a != a) ? a : b; }
  __device__ double kkt_node(const T (&x)[D], const T (&xl)[D], const T (&p)[D], const T (&pr)[D],
                             double delta, double, bool r3) const {
    if constexpr (sizeof(T) == 4) {
      float a[3], J[9];
      {
        float sps, cps, sth, cth, sph, cph;
        sincosf(x[3], &sps, &cps);
        sincosf(x[4], &sth, &cth);
        sincosf(x[5], &sph, &cph);
        const float cc = cph * cps, cs = cph * sps, sc = sph * cps, ss = sph * sps;
        a[0] = ss + cc * sth;
        a[1] = -sc + cs * sth;
        a[2] = cth * cph;
        J[0] = sc - cs * sth; J[1] = cc * cth;   J[2] = cs - sc * sth;
        J[3] = ss + cc * sth; J[4] = cs * cth;   J[5] = -cc - ss * sth;
        J[6] = 0.0f;          J[7] = -sth * cph; J[8] = -cth * sph;
      }
      const float dt = (float)delta;
      const float q6 = p[6], q7 = p[7], q8 = p[8];
      const float u0m = (a[0] * q6 + a[1] * q7 + a[2] * q8) * m_inv * m_inv;   // u0 / m
      const float coef = ah + u0m;
      float r = 0.0f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float pk = p[k];
        float gp;
        if (k < 6) gp = x[6 + k];
        else if (k < 9) gp = ah * a[k - 6] - (k == 8 ? gz : 0.0f) + a[k - 6] * u0m;
        else gp = pk;
        gp += eps * pk;
        r = max_keep_nan(r, fabsf((x[k] - xl[k]) - dt * gp));
        if (r3) {
          float gx;
          if (k < 3) gx = 0.0f;
          else if (k < 6) gx = coef * (J[k - 3] * q6 + J[k] * q7 + J[k + 3] * q8);
          else gx = p[k - 6];
          r = max_keep_nan(r, fabsf((pr[k] - pk) + dt * gx));
        }
      }
      return (double)r;
    } else {
      double a[3], J[9];
      thrust<double>((double)x[3], (double)x[4], (double)x[5], a, J);
      const double q6 = (double)p[6], q7 = (double)p[7], q8 = (double)p[8];
      const double u0 = (a[0] * q6 + a[1] * q7 + a[2] * q8) / m64;
      const double coef = ah64 + u0 / m64;
      double r = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double pk = (double)p[k];
        double gp;
        if (k < 6) gp = (double)x[6 + k];
        else if (k < 9) gp = ah64 * a[k - 6] - (k == 8 ? gz64 : 0.0) + a[k - 6] * u0 / m64;
        else gp = pk;
        gp += eps64 * pk;
        r = max_nan(r, fabs((double)x[k] - (double)xl[k] - delta * gp));
        if (r3) {
          double gx;
          if (k < 3) gx = 0.0;
          else if (k < 6) gx = coef * (J[k - 3] * q6 + J[k] * q7 + J[k + 3] * q8);
          else gx = (double)p[k - 6];
          r = max_nan(r, fabs((double)pr[k] - pk + delta * gx));
        }
      }
      return r;
    }
  }
};

// ---------------------------------------------------------------- tanh drift, small D
// H = <p, tanh(A x)> + |p|^2/2; A is held in shared memory (broadcast reads).
template <typename T, int D>
struct FamTanhDrift {
  static constexpr bool kHasGradX = true;
  static constexpr bool kGame = false;
  static constexpr bool kTimeDep = false;
  struct Shared { T A[D * D]; };
  struct Ctx { T a[D]; };
  const T* A;
  const double* A64;
  __device__ static void load_shared(const SolveArgs<T>& s, Shared& sh) {
    for (int i = threadIdx.x; i < D * D; i += blockDim.x) sh.A[i] = s.A[i];
  }
  __device__ FamTanhDrift(const SolveArgs<T>& s, const Shared& sh) : A(sh.A), A64(s.A64) {}
  __device__ __forceinline__ void context(const T (&x)[D], Ctx& c) const {
#pragma unroll
    for (int i = 0; i < D; ++i) {
      T y = T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) y += A[i * D + k] * x[k];
      c.a[i] = tanh_t<T>(y);
    }
  }
  struct PC { T lam, s; };
  __device__ __forceinline__ PC point(T lam) const { return PC{lam, T(1) / (T(1) + lam)}; }
  __device__ __forceinline__ void prox(const Ctx& c, const PC& pc, const T (&)[D],
                                       T (&v)[D]) const {
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = (v[k] - pc.lam * c.a[k]) * pc.s;
  }
  // the drift averaged with the weights: (1 + lam) p = v - lam (wr a(xr) + wl a(xl))
  __device__ __forceinline__ void prox_mix(const Ctx& cr, const Ctx& cl, const PC& pc, T wr, T wl,
                                           const T (&)[D], const T (&)[D], T (&v)[D]) const {
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = (v[k] - pc.lam * (wr * cr.a[k] + wl * cl.a[k])) * pc.s;
  }
  // Hopf form, node 1 (hs = sigma / W^2, hc = sigma c):
  //   (1 + lam + hs_k) p_k = v_k - hc_k - lam a_k.
  __device__ __forceinline__ void prox_first(const Ctx& c, const PC& pc, const T (&)[D],
                                             T (&v)[D], const T* hs, const T* hc) const {
#pragma unroll
    for (int k = 0; k < D; ++k)
      v[k] = fdiv<T>(v[k] - hc[k] - pc.lam * c.a[k], T(1) + pc.lam + hs[k]);
  }
  __device__ __forceinline__ void gradx(const Ctx& c, const T (&)[D], const T (&p)[D],
                                        T (&g)[D]) const {
    T w[D];
#pragma unroll
    for (int k = 0; k < D; ++k) w[k] = (T(1) - c.a[k] * c.a[k]) * p[k];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) s += A[k * D + i] * w[k];
      g[i] = s;
    }
  }
  __device__ __forceinline__ double H64(const T (&x)[D], const T (&p)[D]) const {
    double h = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      double y = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) y += A64[i * D + k] * (double)x[k];
      const double pi = (double)p[i];
      h += pi * tanh(y) + 0.5 * pi * pi;
    }
    return h;
  }
  __device__ __forceinline__ T Ht(const T (&x)[D], const T (&p)[D]) const {
    T h = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      T y = T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) y += A[i * D + k] * x[k];
      h += p[i] * tanh_t<T>(y) + T(0.5) * p[i] * p[i];
    }
    return h;
  }
  // grad_p H = tanh(A x) + p, grad_x H = A^T ((1 - tanh(A x)^2) p), A in FP64
  __device__ double kkt_node(const T (&x)[D], const T (&xl)[D], const T (&p)[D], const T (&pr)[D],
                             double delta, double, bool r3) const {
    double w[D];
    double r = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      double y = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) y += A64[i * D + k] * (double)x[k];
      const double av = tanh(y), pi = (double)p[i];
      r = max_nan(r, fabs((double)x[i] - (double)xl[i] - delta * (av + pi)));
      w[i] = (1.0 - av * av) * pi;
    }
    if (r3) {
#pragma unroll
      for (int i = 0; i < D; ++i) {
        double g = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) g += A64[k * D + i] * w[k];
        r = max_nan(r, fabs((double)pr[i] - (double)p[i] + delta * g));
      }
    }
    return r;
  }
};

// ---------------------------------------------------------------- eikonal, small D
// H = c(x) |p|_2 with c(x) = c0 + c1 exp(-c2 |x - x_b|^2) (Section 6.1).  The
// dual step is the shrink_2 operator, p = v max(|v| - lam c, 0) / |v|, and
// grad_x H = |p| grad c(x) = |p| (-2 c1 c2 e) (x - x_b), e = exp(-c2 |x - x_b|^2).
// MOVING: the bump moves with velocity v_b, c(x - s v_b) at the node time s
// (Section 6.1's state-and-time-dependent example); the kernel then calls the
// time-aware members (context_t, Ht_t, H64_t) with s = j delta.
template <typename T, int D, bool MOVING>
struct FamEikonalT {
  static constexpr bool kHasGradX = true;
  static constexpr bool kGame = false;
  static constexpr bool kTimeDep = MOVING;
  struct Shared { T xb[D]; T vb[MOVING ? D : 1]; };
  struct CtxS { T c, gf; };                // c(x) and -2 c1 c2 e at x^k
  struct CtxM { T c, gf, s; };             // and the node time
  using Ctx = typename std::conditional<MOVING, CtxM, CtxS>::type;
  struct PC { T lam; };
  const T* xb;
  const T* vb;
  const double* xb64;
  const double* vb64;
  T c0, c1, c2;
  double c0d, c1d, c2d;
  __device__ static void load_shared(const SolveArgs<T>& s, Shared& sh) {
    for (int i = threadIdx.x; i < D; i += blockDim.x) {
      sh.xb[i] = s.xb[i];
      if constexpr (MOVING) sh.vb[i] = s.vb[i];
    }
  }
  __device__ FamEikonalT(const SolveArgs<T>& s, const Shared& sh)
      : xb(sh.xb), vb(sh.vb), xb64(s.xb64), vb64(s.vb64), c0(s.eik_t[0]), c1(s.eik_t[1]),
        c2(s.eik_t[2]), c0d(s.eik_c0), c1d(s.eik_c1), c2d(s.eik_c2) {}
  __device__ __forceinline__ PC point(T lam) const { return PC{lam}; }
  // the bump centre at time s
  __device__ __forceinline__ T centre(int k, T s) const {
    if constexpr (MOVING) return xb[k] + s * vb[k];
    else return xb[k];
  }
  __device__ __forceinline__ void context_t(const T (&x)[D], T s, Ctx& c) const {
    T r2 = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) { const T y = x[k] - centre(k, s); r2 += y * y; }
    const T e = exp_t<T>(-c2 * r2);
    c.c = c0 + c1 * e;
    c.gf = T(-2) * c1 * c2 * e;
    if constexpr (MOVING) c.s = s;
  }
  __device__ __forceinline__ void context(const T (&x)[D], Ctx& c) const { context_t(x, T(0), c); }
  __device__ __forceinline__ void prox(const Ctx& c, const PC& pc, const T (&)[D],
                                       T (&v)[D]) const {
    T n2 = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) n2 += v[k] * v[k];
    const T n = sqrt_t<T>(n2), th = pc.lam * c.c;
    const T keep = (n > th) ? fdiv<T>(n - th, n) : T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] *= keep;
  }
  // shrink_2 with the weighted speed wr c(xr) + wl c(xl)
  __device__ __forceinline__ void prox_mix(const Ctx& cr, const Ctx& cl, const PC& pc, T wr, T wl,
                                           const T (&)[D], const T (&)[D], T (&v)[D]) const {
    T n2 = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) n2 += v[k] * v[k];
    const T n = sqrt_t<T>(n2), th = pc.lam * (wr * cr.c + wl * cl.c);
    const T keep = (n > th) ? fdiv<T>(n - th, n) : T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] *= keep;
  }
  __device__ __forceinline__ void gradx(const Ctx& c, const T (&x)[D], const T (&p)[D],
                                        T (&g)[D]) const {
    T n2 = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) n2 += p[k] * p[k];
    const T sc = sqrt_t<T>(n2) * c.gf;
    T s = T(0);
    if constexpr (MOVING) s = c.s;
#pragma unroll
    for (int k = 0; k < D; ++k) g[k] = sc * (x[k] - centre(k, s));
  }
  __device__ __forceinline__ double H64_t(const T (&x)[D], const T (&p)[D], double s) const {
    double r2 = 0.0, n2 = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double cb = MOVING ? xb64[k] + s * vb64[k] : xb64[k];
      const double y = (double)x[k] - cb;
      r2 += y * y;
      n2 += (double)p[k] * (double)p[k];
    }
    return (c0d + c1d * exp(-c2d * r2)) * sqrt(n2);
  }
  __device__ __forceinline__ double H64(const T (&x)[D], const T (&p)[D]) const {
    return H64_t(x, p, 0.0);
  }
  __device__ __forceinline__ T Ht_t(const T (&x)[D], const T (&p)[D], T s) const {
    Ctx c;
    context_t(x, s, c);
    T n2 = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) n2 += p[k] * p[k];
    return c.c * sqrt_t<T>(n2);
  }
  __device__ __forceinline__ T Ht(const T (&x)[D], const T (&p)[D]) const { return Ht_t(x, p, T(0)); }
  // grad_p H = c(x) p / |p| (for p = 0: r1 is the distance of x_j - x_{j-1} to the
  // ball of radius delta c(x_j), delta times the subdifferential), grad_x H = |p| grad c
  __device__ double kkt_node(const T (&x)[D], const T (&xl)[D], const T (&p)[D], const T (&pr)[D],
                             double delta, double s, bool r3) const {
    double r2 = 0.0, n2 = 0.0, d2 = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double cb = MOVING ? xb64[k] + s * vb64[k] : xb64[k];
      const double y = (double)x[k] - cb, pk = (double)p[k], dk = (double)x[k] - (double)xl[k];
      r2 += y * y;
      n2 += pk * pk;
      d2 += dk * dk;
    }
    const double e = exp(-c2d * r2), c = c0d + c1d * e, gf = -2.0 * c1d * c2d * e;
    const double n = sqrt(n2);
    const double out = n2 > 0.0 ? 0.0 : fmax(0.0, 1.0 - delta * c / (d2 > 0.0 ? sqrt(d2) : 1.0));
    double r = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double pk = (double)p[k], dk = (double)x[k] - (double)xl[k];
      r = max_nan(r, fabs(n2 > 0.0 ? dk - delta * c * pk / n : dk * out));
      if (r3) {
        const double cb = MOVING ? xb64[k] + s * vb64[k] : xb64[k];
        r = max_nan(r, fabs((double)pr[k] - pk + delta * n * gf * ((double)x[k] - cb)));
      }
    }
    return r;
  }
};
template <typename T, int D>
using FamEikonal = FamEikonalT<T, D, false>;
template <typename T, int D>
using FamEikonalMoving = FamEikonalT<T, D, true>;

// ---------------------------------------------------------------- difference-of-norms game
// Section 6.2's differential game: state z = (x, y), x = z[0..d1) (the
// minimising player), y = z[d1..D) (the maximising one); the costate array holds
// (p, q).  H(z, p, q) = c1(z)|p| - c2(z)|q| with c1(z) = c0 + a exp(-b |z - z_b|^2)
// and its mirror c2(z) = c1(-z).  Both dual steps are shrink_2 (thresholds
// lam c1 and lam c2); the primal step is game_step: a descent step for x at z^k,
// then an ascent step for y at (x^{k+1}, y^k) (Algorithm 3's order).
template <typename T, int D>
struct FamGame {
  static constexpr bool kHasGradX = true;
  static constexpr bool kGame = true;
  static constexpr bool kTimeDep = false;
  struct Shared { T zb[D]; };
  struct Ctx { T c1, c2, g1, g2; };        // speeds and gradient factors -2 a b e at z^k
  struct PC { T lam; };
  const T* zb;
  const double* zb64;
  int d1;
  T c0, am, bw;
  double c0d, amd, bwd;
  __device__ static void load_shared(const SolveArgs<T>& s, Shared& sh) {
    for (int i = threadIdx.x; i < D; i += blockDim.x) sh.zb[i] = s.xb[i];
  }
  __device__ FamGame(const SolveArgs<T>& s, const Shared& sh)
      : zb(sh.zb), zb64(s.xb64), d1(s.game_d1), c0(s.eik_t[0]), am(s.eik_t[1]),
        bw(s.eik_t[2]), c0d(s.eik_c0), amd(s.eik_c1), bwd(s.eik_c2) {}
  __device__ __forceinline__ PC point(T lam) const { return PC{lam}; }
  __device__ __forceinline__ void context(const T (&z)[D], Ctx& c) const {
    T r1 = T(0), r2 = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const T u = z[k] - zb[k], w = z[k] + zb[k];
      r1 += u * u;
      r2 += w * w;
    }
    const T e1 = exp_t<T>(-bw * r1), e2 = exp_t<T>(-bw * r2);
    c.c1 = c0 + am * e1;
    c.c2 = c0 + am * e2;
    c.g1 = T(-2) * am * bw * e1;
    c.g2 = T(-2) * am * bw * e2;
  }
  __device__ __forceinline__ void norms(const T (&P)[D], T& np, T& nq) const {
    T sp = T(0), sq = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (k < d1) sp += P[k] * P[k];
      else sq += P[k] * P[k];
    }
    np = sqrt_t<T>(sp);
    nq = sqrt_t<T>(sq);
  }
  __device__ __forceinline__ void prox(const Ctx& c, const PC& pc, const T (&)[D],
                                       T (&v)[D]) const {
    T np, nq;
    norms(v, np, nq);
    const T tp = pc.lam * c.c1, tq = pc.lam * c.c2;
    const T kp = (np > tp) ? fdiv<T>(np - tp, np) : T(0);
    const T kq = (nq > tq) ? fdiv<T>(nq - tq, nq) : T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] *= (k < d1) ? kp : kq;
  }
  // shrink_2 of both players with the weighted speeds (forward-Euler and
  // trapezoid schemes): thresholds lam (wr c_i(zr) + wl c_i(zl))
  __device__ __forceinline__ void prox_mix(const Ctx& cr, const Ctx& cl, const PC& pc, T wr, T wl,
                                           const T (&)[D], const T (&)[D], T (&v)[D]) const {
    T np, nq;
    norms(v, np, nq);
    const T tp = pc.lam * (wr * cr.c1 + wl * cl.c1), tq = pc.lam * (wr * cr.c2 + wl * cl.c2);
    const T kp = (np > tp) ? fdiv<T>(np - tp, np) : T(0);
    const T kq = (nq > tq) ? fdiv<T>(nq - tq, nq) : T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] *= (k < d1) ? kp : kq;
  }
  // xn holds z - tau (P - P_next) on entry
  __device__ __forceinline__ void game_step(const Ctx& c, const T (&z)[D], const T (&P)[D],
                                            T taud, T (&xn)[D]) const {
    T np, nq;
    norms(P, np, nq);
    game_step_norms(c, z, np, nq, taud, xn);
  }
  // grad_z H(z, P) = |p| grad c1(z) - |q| grad c2(z) is linear in the two norms,
  // so a weighted sum of gradients over costates is this step with weighted norms
  __device__ __forceinline__ void game_step_norms(const Ctx& c, const T (&z)[D], T np, T nq,
                                                  T taud, T (&xn)[D]) const {
    const T f1 = np * c.g1, f2 = nq * c.g2;
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (k < d1) xn[k] += taud * (f1 * (z[k] - zb[k]) - f2 * (z[k] + zb[k]));
    T zm[D];
#pragma unroll
    for (int k = 0; k < D; ++k) zm[k] = (k < d1) ? xn[k] : z[k];
    Ctx cm;
    context(zm, cm);
    const T h1 = np * cm.g1, h2 = nq * cm.g2;
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (k >= d1) xn[k] -= taud * (h1 * (zm[k] - zb[k]) - h2 * (zm[k] + zb[k]));
  }
  __device__ __forceinline__ void gradx(const Ctx&, const T (&)[D], const T (&)[D],
                                        T (&g)[D]) const {
#pragma unroll
    for (int k = 0; k < D; ++k) g[k] = T(0);      // the primal step is game_step
  }
  // Node 0 under the mixed schemes, all coordinates: x_0 <- prox of g_x at
  // x_0 + tau p_1 + tau delta wl d_x H(z_0, P_1), then, at m_0 = (x_0^{k+1}, y_0),
  // y_0 <- ascent prox of g_y at y_0 + tau q_1 - tau delta wl d_y H(m_0, P_1)
  // (the prox as offset and reciprocal per coordinate, the maximiser's with -W^2).
  __device__ __forceinline__ void node0_step_mix(const T (&z0)[D], const T (&P1)[D], T tau,
                                                 T taudw, const T* goff, const T* ginv,
                                                 T (&zn)[D]) const {
    T np, nq;
    norms(P1, np, nq);
    Ctx c;
    context(z0, c);
    const T f1 = np * c.g1, f2 = nq * c.g2;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const T gx = f1 * (z0[k] - zb[k]) - f2 * (z0[k] + zb[k]);
      zn[k] = (k < d1) ? (z0[k] + tau * P1[k] + taudw * gx + goff[k]) * ginv[k] : z0[k];
    }
    Ctx cm;
    context(zn, cm);
    const T h1 = np * cm.g1, h2 = nq * cm.g2;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const T gy = h1 * (zn[k] - zb[k]) - h2 * (zn[k] + zb[k]);
      if (k >= d1) zn[k] = (z0[k] + tau * P1[k] - taudw * gy + goff[k]) * ginv[k];
    }
  }
  __device__ __forceinline__ double H64(const T (&z)[D], const T (&P)[D]) const {
    double r1 = 0.0, r2 = 0.0, sp = 0.0, sq = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double u = (double)z[k] - zb64[k], w = (double)z[k] + zb64[k];
      r1 += u * u;
      r2 += w * w;
      const double pk = (double)P[k];
      if (k < d1) sp += pk * pk;
      else sq += pk * pk;
    }
    return (c0d + amd * exp(-bwd * r1)) * sqrt(sp) - (c0d + amd * exp(-bwd * r2)) * sqrt(sq);
  }
  __device__ __forceinline__ T Ht(const T (&z)[D], const T (&P)[D]) const {
    Ctx c;
    context(z, c);
    T np, nq;
    norms(P, np, nq);
    return c.c1 * np - c.c2 * nq;
  }
};

}  // namespace hj
