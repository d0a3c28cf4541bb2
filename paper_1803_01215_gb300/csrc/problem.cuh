// Problem handle and solve helpers shared by the C ABI entry points.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <map>
#include <mutex>
#include <utility>

#include "hj_internal.cuh"
#include "hjpdhg.h"

struct hj_problem_s {
  int family = 0, d = 0, device = 0;
  double qc[4] = {0, 0, 0, 0};        // m, a_h, g_z, eps
  bool w_nonzero = true;              // every W_i != 0 (g* finite: the Hopf form)
  double w2max = 0.0;                 // max_i W_i^2 (the concave x_0 prox needs tau w2max < 1)
  double eik[4] = {1, 0, 0, 0};       // eikonal: s, c0, c1, c2; game: d1, c0, a, b
  double w2max_max = 0.0;             // game: max W_i^2 over the maximiser's coordinates
  double* xbd = nullptr;              // [d] eikonal bump centre
  float* xbf = nullptr;
  bool eik_moving = false;            // eikonal bump moving with velocity v_b
  double* vbd = nullptr;              // [d] v_b
  float* vbf = nullptr;
  double* W2 = nullptr;               // [d]  W_i^2
  double* W = nullptr;                // [d]  W_i as given (sign kept for dV/dW)
  double* c = nullptr;                // [d]
  float* Af = nullptr;                // [d][d]
  float* Atf = nullptr;               // [d][d]
  double* Ad = nullptr;               // [d][d]
  double* Atd = nullptr;              // [d][d]
  unsigned long long* counter = nullptr;
  // Launch shapes chosen by hj_autotune / hj_set_launch_shape, keyed by
  // (precision, N); absent keys use the default shape.
  std::map<std::pair<int, int>, hj::WarpConfig> shapes;
  std::mutex mu;
};

namespace hj {
// Residual of the discrete characteristic equations from trajectories (kkt.cu):
// one thread per (point, node) for the register-resident kernel's families and
// dimensions (kkt_node.cu; HJ_ERR_UNSUPPORTED for others), else one CTA per point.
bool kkt_family_supported(int family);
hj_status launch_kkt(const hj_problem_s* p, int64_t B, int32_t N, bool fp64, const double* t,
                     const void* traj_x, const void* traj_p, double* kkt, cudaStream_t s);
template <typename T>
hj_status launch_kkt_nodes(const hj_problem_s* p, int64_t B, int32_t N, const double* t,
                           const T* X, const T* P, double* kkt, cudaStream_t s);
}  // namespace hj

namespace hj_detail {

inline bool all_finite(const double* v, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

template <typename T>
hj_status upload(T** dst, const T* src, size_t n) {
  if (cudaMalloc(reinterpret_cast<void**>(dst), n * sizeof(T)) != cudaSuccess) return HJ_ERR_OOM;
  if (cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return HJ_ERR_CUDA;
  return HJ_OK;
}

inline void release(hj_problem_s* p) {
  cudaFree(p->W2); cudaFree(p->W); cudaFree(p->c);
  cudaFree(p->Af); cudaFree(p->Atf); cudaFree(p->Ad); cudaFree(p->Atd);
  cudaFree(p->xbd); cudaFree(p->xbf);
  cudaFree(p->vbd); cudaFree(p->vbf);
  cudaFree(p->counter);
  delete p;
}

inline hj::WarpConfig shape_for(hj_problem_s* p, int precision, int N) {
  {
    std::lock_guard<std::mutex> g(p->mu);
    auto it = p->shapes.find({precision, N});
    if (it != p->shapes.end()) return it->second;
  }
  return hj::default_warp_config(p->family, p->d, N, precision == HJ_PREC_FP64);
}

// Which kernel serves a request: the register-resident warp kernel when it has
// an instantiation for (family, d), else the shared-memory CTA kernel (tanh
// drift at any d, or H = |p|^2/2 at any d).
template <typename T>
hj_status dispatch(hj_problem_s* p, const hj::SolveArgs<T>& a, hj::WarpConfig cfg,
                   cudaStream_t s) {
  if (cfg.G > 0) {
    const hj_status r = hj::launch_warp_solver<T>(p->family, a, cfg, s);
    if (r != HJ_ERR_UNSUPPORTED) return r;
  }
  if (a.value_stop) return HJ_ERR_UNSUPPORTED;   // the value test: register kernel only
  if (p->family == HJ_FAMILY_TANH_DRIFT) return hj::launch_td_cta_solver<T>(a, true, s);
  if (p->family == HJ_FAMILY_EIKONAL)
    return a.eik_moving ? HJ_ERR_UNSUPPORTED : hj::launch_eik_cta_solver<T>(a, s);
  if (p->family == HJ_FAMILY_GAME_NORMS) return HJ_ERR_UNSUPPORTED;   // register kernel only
  if (p->family == HJ_FAMILY_QUADRATIC) return hj::launch_td_cta_solver<T>(a, false, s);
  return HJ_ERR_UNSUPPORTED;
}

template <typename T>
void fill_args(hj::SolveArgs<T>& a, const hj_problem_s* prob, int64_t B, int32_t N,
               const hj_solver_opts& o, const double* xq, const double* t, double* V,
               int32_t* iters, int8_t* status, void* traj_x, void* traj_p,
               const void* warm_x, const void* warm_p);

template <>
inline void fill_args<float>(hj::SolveArgs<float>& a, const hj_problem_s* prob, int64_t B, int32_t N,
                      const hj_solver_opts& o, const double* xq, const double* t, double* V,
                      int32_t* iters, int8_t* status, void* traj_x, void* traj_p,
                      const void* warm_x, const void* warm_p) {
  a.A = prob->Af; a.At = prob->Atf; a.xb = prob->xbf; a.vb = prob->vbf;
  a.traj_x = static_cast<float*>(traj_x); a.traj_p = static_cast<float*>(traj_p);
  a.warm_x = static_cast<const float*>(warm_x); a.warm_p = static_cast<const float*>(warm_p);
  (void)B; (void)N; (void)o; (void)xq; (void)t; (void)V; (void)iters; (void)status;
}

template <>
inline void fill_args<double>(hj::SolveArgs<double>& a, const hj_problem_s* prob, int64_t B, int32_t N,
                       const hj_solver_opts& o, const double* xq, const double* t, double* V,
                       int32_t* iters, int8_t* status, void* traj_x, void* traj_p,
                       const void* warm_x, const void* warm_p) {
  a.A = prob->Ad; a.At = prob->Atd; a.xb = prob->xbd; a.vb = prob->vbd;
  a.traj_x = static_cast<double*>(traj_x); a.traj_p = static_cast<double*>(traj_p);
  a.warm_x = static_cast<const double*>(warm_x); a.warm_p = static_cast<const double*>(warm_p);
  (void)B; (void)N; (void)o; (void)xq; (void)t; (void)V; (void)iters; (void)status;
}

template <typename T>
hj::SolveArgs<T> make_args(const hj_problem_s* prob, int64_t B, int32_t N,
                           const hj_solver_opts& o, const double* xq, const double* t,
                           double* V, int32_t* iters, int8_t* status, void* traj_x,
                           void* traj_p, const void* warm_x, const void* warm_p) {
  hj::SolveArgs<T> a{};
  a.B = B; a.N = N; a.d = prob->d;
  a.sigma = o.sigma; a.tau = o.tau; a.theta = o.theta; a.tol = o.tol;
  a.tol_hi = (float)o.tol;
  a.tol_lo = (float)(o.tol - (double)a.tol_hi);
  a.sigma_t = T(o.sigma); a.tau_t = T(o.tau); a.theta_t = T(o.theta);
  a.max_iter = o.max_iter; a.check_every = o.check_every; a.inner_steps = o.inner_steps;
  a.seed = o.seed; a.radius = o.init_radius; a.point_offset = o.point_offset;
  a.formulation = o.formulation;
  // H independent of x (quadratic family): both ends of an interval give the
  // same H, so every scheme is the backward-Euler problem and runs as such
  a.scheme = prob->family == HJ_FAMILY_QUADRATIC ? HJ_SCHEME_BE : o.scheme;
  a.mix_wr = a.scheme == HJ_SCHEME_BE ? 1.0 : (a.scheme == HJ_SCHEME_FE ? 0.0 : 0.5);
  a.mix_wl = 1.0 - a.mix_wr;
  a.mix_wr_t = T(a.mix_wr); a.mix_wl_t = T(a.mix_wl);
  a.value_tol = o.value_tol;
  a.value_stop = o.value_tol > 0.0 ? 1 : 0;
  a.xq = xq; a.t = t; a.V = V; a.iters = iters; a.status = status;
  a.W2 = prob->W2; a.c = prob->c; a.A64 = prob->Ad;
  a.qc_m = prob->qc[0]; a.qc_ah = prob->qc[1]; a.qc_gz = prob->qc[2]; a.qc_eps = prob->qc[3];
  a.eik_c0 = prob->eik[1]; a.eik_c1 = prob->eik[2]; a.eik_c2 = prob->eik[3];
  hj::fill_family_consts(a);
  a.xb64 = prob->xbd;
  a.vb64 = prob->vbd;
  a.eik_moving = prob->eik_moving ? 1 : 0;
  a.cost_sign = (prob->family == HJ_FAMILY_EIKONAL && prob->eik[0] < 0) ? -1.0 : 1.0;
  a.game_d1 = (prob->family == HJ_FAMILY_GAME_NORMS) ? (int32_t)prob->eik[0] : prob->d;
  a.counter = prob->counter;
  a.budget_ns = (int64_t)(o.time_budget_ms * 1e6);
  a.iter_budget = o.iter_budget;
  fill_args<T>(a, prob, B, N, o, xq, t, V, iters, status, traj_x, traj_p, warm_x, warm_p);
  return a;
}

inline hj_status check_opts(const hj_solver_opts& o) {
  if (!(std::isfinite(o.sigma) && o.sigma > 0) || !(std::isfinite(o.tau) && o.tau > 0))
    return HJ_ERR_INVALID_ARG;
  if (!(o.theta >= 0.0 && o.theta <= 1.0) || !(o.tol >= 0.0) || !std::isfinite(o.tol))
    return HJ_ERR_INVALID_ARG;
  if (o.max_iter < 1 || o.check_every < 1 || o.inner_steps < 1) return HJ_ERR_INVALID_ARG;
  if (o.precision != HJ_PREC_FP32 && o.precision != HJ_PREC_FP64) return HJ_ERR_INVALID_ARG;
  if (o.formulation != HJ_FORM_LAX && o.formulation != HJ_FORM_HOPF) return HJ_ERR_INVALID_ARG;
  if (o.scheme != HJ_SCHEME_BE && o.scheme != HJ_SCHEME_FE && o.scheme != HJ_SCHEME_TRAP)
    return HJ_ERR_INVALID_ARG;
  if (!(o.value_tol >= 0.0) || !std::isfinite(o.value_tol)) return HJ_ERR_INVALID_ARG;
  if (!(o.time_budget_ms >= 0.0) || !(o.time_budget_ms <= 9.0e12) || o.iter_budget < 0)
    return HJ_ERR_INVALID_ARG;
  if (!(std::isfinite(o.init_radius) && o.init_radius >= 0.0) || o.point_offset < 0)
    return HJ_ERR_INVALID_ARG;
  if (4.0 * o.sigma * o.tau >= 1.0) return HJ_ERR_STEP_SIZE;
  return HJ_OK;
}

// The Hopf form needs g* finite: every W_i nonzero; the eikonal family is
// solved in the Lax form only, and its negative equation's concave x_0 prox
// needs tau W_i^2 < 1.
inline hj_status check_formulation(const hj_problem_s* p, const hj_solver_opts& o) {
  // the value test: the backward-Euler Lax form (register kernel, checked at dispatch)
  if (o.value_tol > 0.0 && (o.formulation != HJ_FORM_LAX ||
                            (o.scheme != HJ_SCHEME_BE && p->family != HJ_FAMILY_QUADRATIC)))
    return HJ_ERR_UNSUPPORTED;
  // the forward-Euler and trapezoid forms: Lax form, one gradient step
  if (o.scheme != HJ_SCHEME_BE && p->family != HJ_FAMILY_QUADRATIC &&
      (o.formulation != HJ_FORM_LAX || o.inner_steps != 1))
    return HJ_ERR_UNSUPPORTED;
  if (o.formulation == HJ_FORM_HOPF && p->family == HJ_FAMILY_EIKONAL) return HJ_ERR_UNSUPPORTED;
  // a moving bump: backward-Euler Lax form (the register kernel)
  if (p->eik_moving && o.scheme != HJ_SCHEME_BE) return HJ_ERR_UNSUPPORTED;
  if (o.formulation == HJ_FORM_HOPF && !p->w_nonzero) return HJ_ERR_INVALID_ARG;
  if (p->family == HJ_FAMILY_EIKONAL && p->eik[0] < 0 && !(o.tau * p->w2max < 1.0))
    return HJ_ERR_STEP_SIZE;
  if (p->family == HJ_FAMILY_GAME_NORMS) {
    if (o.formulation != HJ_FORM_LAX || o.inner_steps != 1) return HJ_ERR_UNSUPPORTED;
    if (!(o.tau * p->w2max_max < 1.0)) return HJ_ERR_STEP_SIZE;
  }
  return HJ_OK;
}

template <typename T>
hj_status run_solve(hj_problem_s* prob, int64_t B, int32_t N, const hj_solver_opts& o,
                    hj::WarpConfig cfg, const double* xq, const double* t, double* V,
                    int32_t* iters, int8_t* status, void* traj_x, void* traj_p,
                    const void* warm_x, const void* warm_p, cudaStream_t s) {
  if (cudaMemsetAsync(prob->counter, 0, hj::kCounterWords * sizeof(unsigned long long), s) !=
      cudaSuccess)
    return HJ_ERR_CUDA;
  const hj::SolveArgs<T> a = make_args<T>(prob, B, N, o, xq, t, V, iters, status, traj_x,
                                          traj_p, warm_x, warm_p);
  return dispatch<T>(prob, a, cfg, s);
}

// The solve with the per-point residual of the discrete characteristic
// equations, evaluated after the solve from the trajectories (written to a
// stream-ordered workspace when the caller passes none).
template <typename T>
hj_status run_solve_kkt(hj_problem_s* prob, int64_t B, int32_t N, const hj_solver_opts& o,
                        hj::WarpConfig cfg, const double* xq, const double* t, double* V,
                        int32_t* iters, int8_t* status, double* kkt, void* traj_x, void* traj_p,
                        const void* warm_x, const void* warm_p, cudaStream_t s) {
  const size_t bytes = (size_t)B * (size_t)(N + 1) * (size_t)prob->d * sizeof(T);
  unsigned char* ws = nullptr;
  const int need = (traj_x == nullptr) + (traj_p == nullptr);
  if (need > 0 && cudaMallocAsync(reinterpret_cast<void**>(&ws), need * bytes, s) != cudaSuccess)
    return HJ_ERR_OOM;
  void* tx = traj_x != nullptr ? traj_x : ws;
  void* tp = traj_p != nullptr ? traj_p : (traj_x != nullptr ? ws : ws + bytes);
  hj_status r = run_solve<T>(prob, B, N, o, cfg, xq, t, V, iters, status, tx, tp, warm_x, warm_p, s);
  if (r == HJ_OK) r = hj::launch_kkt(prob, B, N, sizeof(T) == 8, t, tx, tp, kkt, s);
  if (ws != nullptr && cudaFreeAsync(ws, s) != cudaSuccess && r == HJ_OK) r = HJ_ERR_CUDA;
  return r;
}

}  // namespace hj_detail
