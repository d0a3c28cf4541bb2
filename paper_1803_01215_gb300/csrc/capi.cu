// C ABI of the solver: argument validation, problem handles, kernel dispatch.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "hj_internal.cuh"
#include "hjpdhg.h"

struct hj_problem_s {
  int family = 0, d = 0, device = 0;
  double qc[4] = {0, 0, 0, 0};        // m, a_h, g_z, eps
  double* W2 = nullptr;               // [d]
  double* c = nullptr;                // [d]
  float* Af = nullptr;                // [d][d]
  float* Atf = nullptr;               // [d][d]
  double* Ad = nullptr;               // [d][d]
  double* Atd = nullptr;              // [d][d]
  unsigned long long* counter = nullptr;
};

namespace {

bool all_finite(const double* v, int64_t n) {
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

void release(hj_problem_s* p) {
  cudaFree(p->W2); cudaFree(p->c);
  cudaFree(p->Af); cudaFree(p->Atf); cudaFree(p->Ad); cudaFree(p->Atd);
  cudaFree(p->counter);
  delete p;
}

// Which kernel serves a request: the register-resident warp kernel when it has
// an instantiation for (family, d, N), else the shared-memory tanh-drift kernel.
template <typename T>
hj_status dispatch(const hj_problem_s* p, const hj::SolveArgs<T>& a, cudaStream_t s) {
  hj_status r = hj::launch_warp_solver<T>(p->family, a, s);
  if (r != HJ_ERR_UNSUPPORTED) return r;
  if (p->family == HJ_FAMILY_TANH_DRIFT) return hj::launch_td_cta_solver<T>(a, s);
  return HJ_ERR_UNSUPPORTED;
}

}  // namespace

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

int32_t hj_version(void) { return 100; }

hj_status hj_problem_create(hj_problem* out, int32_t family, int32_t d, const double* dyn,
                            int64_t n_dyn, const double* W, const double* c) {
  if (out == nullptr) return HJ_ERR_INVALID_ARG;
  *out = nullptr;
  if (d < 1 || d > hj::kMaxD || W == nullptr || c == nullptr || n_dyn < 0)
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
    default:
      return HJ_ERR_INVALID_ARG;
  }
  if (!all_finite(W, d) || !all_finite(c, d) || (n_dyn > 0 && !all_finite(dyn, n_dyn)))
    return HJ_ERR_INVALID_ARG;

  hj_problem_s* p = new (std::nothrow) hj_problem_s();
  if (p == nullptr) return HJ_ERR_OOM;
  p->family = family;
  p->d = d;
  if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return HJ_ERR_CUDA; }
  std::vector<double> w2(d);
  for (int i = 0; i < d; ++i) w2[i] = W[i] * W[i];
  hj_status r = upload(&p->W2, w2.data(), d);
  if (r == HJ_OK) r = upload(&p->c, c, d);
  if (r == HJ_OK && family == HJ_FAMILY_QUADCOPTER) {
    for (int i = 0; i < 4; ++i) p->qc[i] = dyn[i];
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
                               sizeof(unsigned long long)) != cudaSuccess)
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
                         int8_t* status, void* traj_x, void* traj_p, const void* warm_x,
                         const void* warm_p, void* stream) {
  if (prob == nullptr || opts == nullptr || B < 0) return HJ_ERR_INVALID_ARG;
  if (N < 1 || N > hj::kMaxN) return HJ_ERR_INVALID_ARG;
  const hj_solver_opts& o = *opts;
  if (!(std::isfinite(o.sigma) && o.sigma > 0) || !(std::isfinite(o.tau) && o.tau > 0))
    return HJ_ERR_INVALID_ARG;
  if (!(o.theta >= 0.0 && o.theta <= 1.0) || !(o.tol >= 0.0) || !std::isfinite(o.tol))
    return HJ_ERR_INVALID_ARG;
  if (o.max_iter < 1 || o.check_every < 1 || o.inner_steps < 1) return HJ_ERR_INVALID_ARG;
  if (o.precision != HJ_PREC_FP32 && o.precision != HJ_PREC_FP64) return HJ_ERR_INVALID_ARG;
  if (!(std::isfinite(o.init_radius) && o.init_radius >= 0.0) || o.point_offset < 0)
    return HJ_ERR_INVALID_ARG;
  if ((warm_x == nullptr) != (warm_p == nullptr)) return HJ_ERR_INVALID_ARG;
  if (o.point_offset + B > (int64_t(1) << 32)) return HJ_ERR_INVALID_ARG;
  if (4.0 * o.sigma * o.tau >= 1.0) return HJ_ERR_STEP_SIZE;
  if (B == 0) return HJ_OK;
  if (xq == nullptr || t == nullptr || V == nullptr || iters == nullptr || status == nullptr)
    return HJ_ERR_INVALID_ARG;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return HJ_ERR_CUDA;
  if (cur != prob->device) return HJ_ERR_INVALID_ARG;

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(prob->counter, 0, sizeof(unsigned long long), s) != cudaSuccess)
    return HJ_ERR_CUDA;
  if (o.precision == HJ_PREC_FP32) {
    hj::SolveArgs<float> a{};
    a.B = B; a.N = N; a.d = prob->d;
    a.sigma = o.sigma; a.tau = o.tau; a.theta = o.theta; a.tol = o.tol;
    a.max_iter = o.max_iter; a.check_every = o.check_every; a.inner_steps = o.inner_steps;
    a.seed = o.seed; a.radius = o.init_radius; a.point_offset = o.point_offset;
    a.xq = xq; a.t = t; a.V = V; a.iters = iters; a.status = status;
    a.traj_x = static_cast<float*>(traj_x); a.traj_p = static_cast<float*>(traj_p);
    a.warm_x = static_cast<const float*>(warm_x); a.warm_p = static_cast<const float*>(warm_p);
    a.W2 = prob->W2; a.c = prob->c; a.A = prob->Af; a.At = prob->Atf; a.A64 = prob->Ad;
    a.qc_m = prob->qc[0]; a.qc_ah = prob->qc[1]; a.qc_gz = prob->qc[2]; a.qc_eps = prob->qc[3];
    a.counter = prob->counter;
    return dispatch<float>(prob, a, s);
  }
  hj::SolveArgs<double> a{};
  a.B = B; a.N = N; a.d = prob->d;
  a.sigma = o.sigma; a.tau = o.tau; a.theta = o.theta; a.tol = o.tol;
  a.max_iter = o.max_iter; a.check_every = o.check_every; a.inner_steps = o.inner_steps;
  a.seed = o.seed; a.radius = o.init_radius; a.point_offset = o.point_offset;
  a.xq = xq; a.t = t; a.V = V; a.iters = iters; a.status = status;
  a.traj_x = static_cast<double*>(traj_x); a.traj_p = static_cast<double*>(traj_p);
  a.warm_x = static_cast<const double*>(warm_x); a.warm_p = static_cast<const double*>(warm_p);
  a.W2 = prob->W2; a.c = prob->c; a.A = prob->Ad; a.At = prob->Atd; a.A64 = prob->Ad;
  a.qc_m = prob->qc[0]; a.qc_ah = prob->qc[1]; a.qc_gz = prob->qc[2]; a.qc_eps = prob->qc[3];
  a.counter = prob->counter;
  return dispatch<double>(prob, a, s);
}

}  // extern "C"
