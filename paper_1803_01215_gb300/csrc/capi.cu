// C ABI of the solver: argument validation, problem handles, kernel dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "hj_internal.cuh"
#include "hjpdhg.h"

#include "problem.cuh"

using namespace hj_detail;

extern "C" {

const char* hj_status_str(hj_status s) {
  switch (s) {
    case HJ_OK: return "ok";
    case HJ_ERR_INVALID_ARG: return "invalid argument";
    case HJ_ERR_UNSUPPORTED: return "unsupported problem size or option";
    case HJ_ERR_STEP_SIZE: return "step sizes violate sigma*tau*4 < 1";
    case HJ_ERR_CUDA: return "CUDA error";
    case HJ_ERR_OOM: return "device allocation failed";
  }
  return "unknown status";
}

int32_t hj_version(void) { return 200; }

hj_status hj_problem_create(hj_problem* out, int32_t family, int32_t d, const double* dyn,
                            int64_t n_dyn, const double* W, const double* c) {
  if (out == nullptr) return HJ_ERR_INVALID_ARG;
  *out = nullptr;
  if (d < 1 || d > (family == HJ_FAMILY_EIKONAL ? hj::kMaxDEik : hj::kMaxD) || W == nullptr ||
      c == nullptr || n_dyn < 0)
    return HJ_ERR_INVALID_ARG;
  if (n_dyn > 0 && dyn == nullptr) return HJ_ERR_INVALID_ARG;
  switch (family) {
    case HJ_FAMILY_QUADRATIC:
      if (n_dyn != 0) return HJ_ERR_INVALID_ARG;
      break;
    case HJ_FAMILY_QUADCOPTER:
      if (d != 12 || n_dyn != 4) return HJ_ERR_INVALID_ARG;
      if (!(dyn[0] > 0.0) || !(dyn[3] >= 0.0)) return HJ_ERR_INVALID_ARG;
      break;
    case HJ_FAMILY_TANH_DRIFT:
      if (n_dyn != (int64_t)d * d) return HJ_ERR_INVALID_ARG;
      break;
    case HJ_FAMILY_GAME_NORMS:
      if (n_dyn != 4 + (int64_t)d || d < 2) return HJ_ERR_INVALID_ARG;
      if (!(dyn[0] >= 1.0 && dyn[0] <= d - 1.0 && dyn[0] == (double)(int)dyn[0]) ||
          !(dyn[1] > 0.0) || !(dyn[2] >= 0.0) || !(dyn[3] >= 0.0))
        return HJ_ERR_INVALID_ARG;
      break;
    case HJ_FAMILY_EIKONAL:
      if (n_dyn != 4 + (int64_t)d && n_dyn != 4 + 2 * (int64_t)d) return HJ_ERR_INVALID_ARG;
      if (!(dyn[0] == 1.0 || dyn[0] == -1.0) || !(dyn[1] > 0.0) || !(dyn[2] >= 0.0) ||
          !(dyn[3] >= 0.0))
        return HJ_ERR_INVALID_ARG;
      break;
    default:
      return HJ_ERR_INVALID_ARG;
  }
  if (!all_finite(W, d) || !all_finite(c, d) || (n_dyn > 0 && !all_finite(dyn, n_dyn)))
    return HJ_ERR_INVALID_ARG;

  hj_problem_s* p = new (std::nothrow) hj_problem_s();
  if (p == nullptr) return HJ_ERR_OOM;
  p->family = family;
  p->d = d;
  for (int i = 0; i < d; ++i) {
    if (W[i] == 0.0) p->w_nonzero = false;
    p->w2max = std::max(p->w2max, W[i] * W[i]);
  }
  if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return HJ_ERR_CUDA; }
  std::vector<double> w2(d);
  for (int i = 0; i < d; ++i) w2[i] = W[i] * W[i];
  hj_status r = upload(&p->W2, w2.data(), d);
  if (r == HJ_OK) r = upload(&p->W, W, d);
  if (r == HJ_OK) r = upload(&p->c, c, d);
  if (r == HJ_OK && family == HJ_FAMILY_QUADCOPTER) {
    for (int i = 0; i < 4; ++i) p->qc[i] = dyn[i];
  }
  if (family == HJ_FAMILY_GAME_NORMS)
    for (int i = (int)dyn[0]; i < d; ++i) p->w2max_max = std::max(p->w2max_max, W[i] * W[i]);
  if (r == HJ_OK && (family == HJ_FAMILY_EIKONAL || family == HJ_FAMILY_GAME_NORMS)) {
    for (int i = 0; i < 4; ++i) p->eik[i] = dyn[i];
    std::vector<float> xf(d);
    for (int i = 0; i < d; ++i) xf[i] = (float)dyn[4 + i];
    r = upload(&p->xbd, dyn + 4, d);
    if (r == HJ_OK) r = upload(&p->xbf, xf.data(), d);
    // eikonal with a moving bump: velocity v_b after x_b (kept only when nonzero)
    bool moving = false;
    if (family == HJ_FAMILY_EIKONAL && n_dyn == 4 + 2 * (int64_t)d)
      for (int i = 0; i < d; ++i) moving = moving || dyn[4 + d + i] != 0.0;
    if (r == HJ_OK && moving) {
      p->eik_moving = true;
      std::vector<float> vf(d);
      for (int i = 0; i < d; ++i) vf[i] = (float)dyn[4 + d + i];
      r = upload(&p->vbd, dyn + 4 + d, d);
      if (r == HJ_OK) r = upload(&p->vbf, vf.data(), d);
    }
  }
  if (r == HJ_OK && family == HJ_FAMILY_TANH_DRIFT) {
    const size_t n = (size_t)d * d;
    std::vector<double> at(n);
    std::vector<float> af(n), atf(n);
    for (int i = 0; i < d; ++i)
      for (int k = 0; k < d; ++k) {
        at[(size_t)k * d + i] = dyn[(size_t)i * d + k];
        af[(size_t)i * d + k] = (float)dyn[(size_t)i * d + k];
        atf[(size_t)k * d + i] = (float)dyn[(size_t)i * d + k];
      }
    r = upload(&p->Ad, dyn, n);
    if (r == HJ_OK) r = upload(&p->Atd, at.data(), n);
    if (r == HJ_OK) r = upload(&p->Af, af.data(), n);
    if (r == HJ_OK) r = upload(&p->Atf, atf.data(), n);
  }
  if (r == HJ_OK && cudaMalloc(reinterpret_cast<void**>(&p->counter),
                               hj::kCounterWords * sizeof(unsigned long long)) != cudaSuccess)
    r = HJ_ERR_OOM;
  if (r != HJ_OK) { release(p); return r; }
  *out = p;
  return HJ_OK;
}

hj_status hj_problem_destroy(hj_problem prob) {
  if (prob == nullptr) return HJ_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(prob->device);
  cudaDeviceSynchronize();
  release(prob);
  cudaSetDevice(cur);
  return HJ_OK;
}

hj_status hj_solve_batch(hj_problem prob, int64_t B, const double* xq, const double* t,
                         int32_t N, const hj_solver_opts* opts, double* V, int32_t* iters,
                         int8_t* status, double* kkt, void* traj_x, void* traj_p,
                         const void* warm_x, const void* warm_p, void* stream) {
  if (prob == nullptr || opts == nullptr || B < 0) return HJ_ERR_INVALID_ARG;
  if (N < 1 || N > hj::kMaxN) return HJ_ERR_INVALID_ARG;
  const hj_solver_opts& o = *opts;
  const hj_status oc = check_opts(o);
  if (oc != HJ_OK) return oc;
  const hj_status fc = check_formulation(prob, o);
  if (fc != HJ_OK) return fc;
  if ((warm_x == nullptr) != (warm_p == nullptr)) return HJ_ERR_INVALID_ARG;
  if (o.point_offset + B > (int64_t(1) << 32)) return HJ_ERR_INVALID_ARG;
  // the residual of the backward-Euler characteristic equations (control and
  // eikonal families; the quadratic family's every scheme is backward Euler)
  if (kkt != nullptr && (!hj::kkt_family_supported(prob->family) ||
                         (o.scheme != HJ_SCHEME_BE && prob->family != HJ_FAMILY_QUADRATIC)))
    return HJ_ERR_UNSUPPORTED;
  if (B == 0) return HJ_OK;
  if (xq == nullptr || t == nullptr || V == nullptr || iters == nullptr || status == nullptr)
    return HJ_ERR_INVALID_ARG;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return HJ_ERR_CUDA;
  if (cur != prob->device) return HJ_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const hj::WarpConfig cfg = shape_for(prob, o.precision, N);
  if (kkt != nullptr) {
    if (o.precision == HJ_PREC_FP32)
      return run_solve_kkt<float>(prob, B, N, o, cfg, xq, t, V, iters, status, kkt, traj_x,
                                  traj_p, warm_x, warm_p, s);
    return run_solve_kkt<double>(prob, B, N, o, cfg, xq, t, V, iters, status, kkt, traj_x,
                                 traj_p, warm_x, warm_p, s);
  }
  if (o.precision == HJ_PREC_FP32)
    return run_solve<float>(prob, B, N, o, cfg, xq, t, V, iters, status, traj_x, traj_p,
                            warm_x, warm_p, s);
  return run_solve<double>(prob, B, N, o, cfg, xq, t, V, iters, status, traj_x, traj_p, warm_x,
                           warm_p, s);
}

hj_status hj_solve_grad(hj_problem prob, int64_t B, const double* t, int32_t N,
                        int32_t precision, const void* traj_x, const void* traj_p,
                        const double* dL_dV, double* dW, double* dc, double* ddyn, double* dxq,
                        void* stream) {
  if (prob == nullptr || B < 0 || N < 1 || N > hj::kMaxN) return HJ_ERR_INVALID_ARG;
  if (precision != HJ_PREC_FP32 && precision != HJ_PREC_FP64) return HJ_ERR_INVALID_ARG;
  if (prob->family == HJ_FAMILY_GAME_NORMS) return HJ_ERR_UNSUPPORTED;
  const int n_dyn = prob->family == HJ_FAMILY_QUADCOPTER ? 4
                    : prob->family == HJ_FAMILY_TANH_DRIFT ? prob->d * prob->d
                    : prob->family == HJ_FAMILY_EIKONAL ? 4 + prob->d * (prob->eik_moving ? 2 : 1)
                    : 0;
  if (dW == nullptr || dc == nullptr || (n_dyn > 0 && ddyn == nullptr)) return HJ_ERR_INVALID_ARG;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return HJ_ERR_CUDA;
  if (cur != prob->device) return HJ_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(dW, 0, prob->d * sizeof(double), s) != cudaSuccess ||
      cudaMemsetAsync(dc, 0, prob->d * sizeof(double), s) != cudaSuccess ||
      (n_dyn > 0 && cudaMemsetAsync(ddyn, 0, n_dyn * sizeof(double), s) != cudaSuccess))
    return HJ_ERR_CUDA;
  if (B == 0) return HJ_OK;
  if (t == nullptr || traj_x == nullptr || traj_p == nullptr || dL_dV == nullptr)
    return HJ_ERR_INVALID_ARG;
  if (precision == HJ_PREC_FP32) {
    hj::GradArgs<float> g{};
    g.B = B; g.N = N; g.d = prob->d; g.n_dyn = n_dyn; g.t = t;
    g.X = static_cast<const float*>(traj_x); g.P = static_cast<const float*>(traj_p);
    g.w = dL_dV; g.W = prob->W; g.W2 = prob->W2; g.c = prob->c; g.A = prob->Af;
    g.qc_m = prob->qc[0]; g.qc_ah = prob->qc[1]; g.qc_gz = prob->qc[2]; g.qc_eps = prob->qc[3];
    g.cost_sign = prob->eik[0] < 0 ? -1.0 : 1.0;
    g.eik_c0 = prob->eik[1]; g.eik_c1 = prob->eik[2]; g.eik_c2 = prob->eik[3];
    g.xb64 = prob->xbd; g.vb64 = prob->vbd;
    g.dW = dW; g.dc = dc; g.ddyn = ddyn; g.dxq = dxq;
    return hj::launch_value_grad<float>(prob->family, g, s);
  }
  hj::GradArgs<double> g{};
  g.B = B; g.N = N; g.d = prob->d; g.n_dyn = n_dyn; g.t = t;
  g.X = static_cast<const double*>(traj_x); g.P = static_cast<const double*>(traj_p);
  g.w = dL_dV; g.W = prob->W; g.W2 = prob->W2; g.c = prob->c; g.A = prob->Ad;
  g.qc_m = prob->qc[0]; g.qc_ah = prob->qc[1]; g.qc_gz = prob->qc[2]; g.qc_eps = prob->qc[3];
  g.cost_sign = prob->eik[0] < 0 ? -1.0 : 1.0;
  g.eik_c0 = prob->eik[1]; g.eik_c1 = prob->eik[2]; g.eik_c2 = prob->eik[3];
  g.xb64 = prob->xbd; g.vb64 = prob->vbd;
  g.dW = dW; g.dc = dc; g.ddyn = ddyn; g.dxq = dxq;
  return hj::launch_value_grad<double>(prob->family, g, s);
}

hj_status hj_solve_grad_unrolled(hj_problem prob, int64_t B, const double* xq, const double* t,
                                 int32_t N, const hj_solver_opts* opts, const int32_t* iters,
                                 int32_t max_iters, int32_t checkpoint_every, const double* dL_dV,
                                 double* dW, double* dc, double* ddyn, double* dxq, void* stream) {
  if (prob == nullptr || opts == nullptr || B < 0 || N < 1 || N > hj::kMaxN) return HJ_ERR_INVALID_ARG;
  const hj_status oc = check_opts(*opts);
  if (oc != HJ_OK) return oc;
  if (max_iters < 0 || checkpoint_every < 1) return HJ_ERR_INVALID_ARG;
  if (opts->inner_steps != 1) return HJ_ERR_UNSUPPORTED;   // one gradient step per x-update
  if (opts->formulation != HJ_FORM_LAX || opts->scheme != HJ_SCHEME_BE)
    return HJ_ERR_UNSUPPORTED;                   // the backward-Euler Lax iteration only
  const bool qc = prob->family == HJ_FAMILY_QUADCOPTER;
  if (!(qc || (prob->family == HJ_FAMILY_QUADRATIC && prob->d <= 4))) return HJ_ERR_UNSUPPORTED;
  if (dW == nullptr || dc == nullptr || dxq == nullptr || (qc && ddyn == nullptr))
    return HJ_ERR_INVALID_ARG;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return HJ_ERR_CUDA;
  if (cur != prob->device) return HJ_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(dW, 0, prob->d * sizeof(double), s) != cudaSuccess ||
      cudaMemsetAsync(dc, 0, prob->d * sizeof(double), s) != cudaSuccess ||
      (qc && cudaMemsetAsync(ddyn, 0, 4 * sizeof(double), s) != cudaSuccess))
    return HJ_ERR_CUDA;
  if (B == 0) return HJ_OK;
  if (xq == nullptr || t == nullptr || iters == nullptr || dL_dV == nullptr)
    return HJ_ERR_INVALID_ARG;
  const bool f64 = opts->precision == HJ_PREC_FP64;
  const size_t tsz = f64 ? sizeof(double) : sizeof(float);
  const int grid = hj::adjoint_grid(B);
  const size_t per_cta = (size_t)(max_iters / checkpoint_every + 1) * 3 * (N + 1) * prob->d * tsz;
  void* work = nullptr;
  if (cudaMalloc(&work, per_cta * grid) != cudaSuccess) return HJ_ERR_OOM;
  if (cudaMemsetAsync(prob->counter, 0, sizeof(unsigned long long), s) != cudaSuccess) {
    cudaFree(work);
    return HJ_ERR_CUDA;
  }
  hj_status r;
  auto fill = [&](auto& a) {
    a.B = B; a.N = N; a.d = prob->d; a.K_cap = max_iters; a.C = checkpoint_every;
    a.radius = opts->init_radius; a.seed = opts->seed; a.point_offset = opts->point_offset;
    a.xq = xq; a.t = t; a.iters = iters; a.w = dL_dV;
    a.W2 = prob->W2; a.W = prob->W; a.c = prob->c;
    a.qc_m = prob->qc[0]; a.qc_ah = prob->qc[1]; a.qc_gz = prob->qc[2]; a.qc_eps = prob->qc[3];
    a.dW = dW; a.dc = dc; a.ddyn = ddyn; a.dxq = dxq; a.counter = prob->counter;
  };
  if (f64) {
    hj::AdjArgs<double> a{};
    fill(a);
    a.sig = opts->sigma; a.tau = opts->tau; a.th = opts->theta;
    a.work = static_cast<double*>(work);
    r = hj::launch_adjoint<double>(prob->family, a, grid, s);
  } else {
    hj::AdjArgs<float> a{};
    fill(a);
    a.sig = (float)opts->sigma; a.tau = (float)opts->tau; a.th = (float)opts->theta;
    a.work = static_cast<float*>(work);
    r = hj::launch_adjoint<float>(prob->family, a, grid, s);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess && r == HJ_OK) r = HJ_ERR_CUDA;
  cudaFree(work);
  return r;
}

hj_status hj_set_launch_shape(hj_problem prob, int32_t precision, int32_t N,
                              int32_t warps_per_point, int32_t nodes_per_lane) {
  if (prob == nullptr || N < 1 || N > hj::kMaxN) return HJ_ERR_INVALID_ARG;
  if (precision != HJ_PREC_FP32 && precision != HJ_PREC_FP64) return HJ_ERR_INVALID_ARG;
  hj::WarpConfig c{warps_per_point, nodes_per_lane};
  if (warps_per_point == 0) c = hj::WarpConfig{1, nodes_per_lane, 1};   // half a warp
  if (!hj::warp_config_available(prob->family, prob->d, c, precision == HJ_PREC_FP64))
    return HJ_ERR_UNSUPPORTED;
  if (N > hj::warp_config_lanes(c) * c.NPL) return HJ_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> g(prob->mu);
  prob->shapes[{precision, N}] = c;
  return HJ_OK;
}

hj_status hj_get_launch_shape(hj_problem prob, int32_t precision, int32_t N,
                              int32_t* warps_per_point, int32_t* nodes_per_lane) {
  if (prob == nullptr || warps_per_point == nullptr || nodes_per_lane == nullptr)
    return HJ_ERR_INVALID_ARG;
  if (N < 1 || N > hj::kMaxN) return HJ_ERR_INVALID_ARG;
  const hj::WarpConfig c = shape_for(prob, precision, N);
  *warps_per_point = c.half ? 0 : c.G;
  *nodes_per_lane = c.NPL;
  return HJ_OK;
}

hj_status hj_autotune(hj_problem prob, int64_t B, const double* xq, const double* t, int32_t N,
                      const hj_solver_opts* opts, int32_t repeats, int32_t* warps_per_point,
                      int32_t* nodes_per_lane, float* best_ms, void* stream) {
  if (prob == nullptr || opts == nullptr || xq == nullptr || t == nullptr || B < 1)
    return HJ_ERR_INVALID_ARG;
  if (N < 1 || N > hj::kMaxN || repeats < 1) return HJ_ERR_INVALID_ARG;
  const hj_status oc = check_opts(*opts);
  if (oc != HJ_OK) return oc;
  const hj_status fc = check_formulation(prob, *opts);
  if (fc != HJ_OK) return fc;
  const bool f64 = opts->precision == HJ_PREC_FP64;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double* V = nullptr;
  int32_t* it = nullptr;
  int8_t* st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hj_status r = HJ_OK;
  if (cudaMalloc(&V, B * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&it, B * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&st, B * sizeof(int8_t)) != cudaSuccess)
    r = HJ_ERR_OOM;
  if (r == HJ_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    r = HJ_ERR_CUDA;
  float best = -1.0f;
  hj::WarpConfig best_c{0, 0};
  const int Gs[5] = {0, 1, 2, 4, 8};             // 0: half a warp
  for (int npl = 1; npl <= 2 && r == HJ_OK; ++npl) {
    for (int gi = 0; gi < 5 && r == HJ_OK; ++gi) {
      const hj::WarpConfig c = Gs[gi] == 0 ? hj::WarpConfig{1, npl, 1} : hj::WarpConfig{Gs[gi], npl};
      if (!hj::warp_config_available(prob->family, prob->d, c, f64) ||
          N > hj::warp_config_lanes(c) * c.NPL)
        continue;
      float tot = 0.0f;
      for (int rep = 0; rep <= repeats && r == HJ_OK; ++rep) {   // rep 0 warms up
        if (cudaEventRecord(e0, s) != cudaSuccess) { r = HJ_ERR_CUDA; break; }
        r = f64 ? run_solve<double>(prob, B, N, *opts, c, xq, t, V, it, st, nullptr, nullptr,
                                    nullptr, nullptr, s)
                : run_solve<float>(prob, B, N, *opts, c, xq, t, V, it, st, nullptr, nullptr,
                                   nullptr, nullptr, s);
        if (r != HJ_OK) break;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
          r = HJ_ERR_CUDA;
          break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tot += ms;
      }
      if (r == HJ_OK && (best < 0.0f || tot / repeats < best)) {
        best = tot / repeats;
        best_c = c;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(V); cudaFree(it); cudaFree(st);
  if (r != HJ_OK) return r;
  if (best_c.G == 0) return HJ_ERR_UNSUPPORTED;
  {
    std::lock_guard<std::mutex> g(prob->mu);
    prob->shapes[{opts->precision, N}] = best_c;
  }
  if (warps_per_point) *warps_per_point = best_c.half ? 0 : best_c.G;
  if (nodes_per_lane) *nodes_per_lane = best_c.NPL;
  if (best_ms) *best_ms = best;
  return HJ_OK;
}

}  // extern "C"
