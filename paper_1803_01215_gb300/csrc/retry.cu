// hj_solve_batch_retry: the batched solve followed by retry rounds for the
// points that reach the iteration cap.
//
// Section 6.2 raises sigma by a fixed step (and sets tau from the step-size
// bound) for game points that hit the maximum count; Section 6.1 reruns such
// points.  Round 0 is hj_solve_batch.  Before round r a small kernel lists the
// points whose status is HJ_POINT_MAX_ITER (order irrelevant: every point is
// solved on its own) and adds their iterations so far to a per-point total;
// round r then launches the same solver kernels on that list (SolveArgs::idx)
// with sigma_r = sigma + r * sigma_step, tau_r = step_product / sigma_r, from a
// fresh initial guess drawn with seed + r or, with warm = 1, from a copy of the
// point's last iterate; with policy value_tol > 0 the last round also applies
// the value test (the paper's switch to a value criterion after a maximum
// count).  Each round reads the list length back to the host.
#include <cuda_runtime.h>

#include <cmath>

#include "hj_internal.cuh"
#include "hjpdhg.h"
#include "problem.cuh"

using namespace hj_detail;

namespace {

// Points still at the cap: appended to idx (atomic slot), iterations banked.
__global__ void collect_capped(const int8_t* status, const int32_t* iters, int64_t B,
                               int32_t* idx, int32_t* count, int32_t* banked) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B;
       b += (int64_t)gridDim.x * blockDim.x) {
    if (status[b] == HJ_POINT_MAX_ITER) {
      idx[atomicAdd(count, 1)] = (int32_t)b;
      banked[b] += iters[b];
    }
  }
}

__global__ void mark_round(const int32_t* idx, int32_t n, int8_t* rounds, int8_t r) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    rounds[idx[i]] = r;
}

__global__ void add_banked(int64_t B, int32_t* iters, const int32_t* banked) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B;
       b += (int64_t)gridDim.x * blockDim.x)
    iters[b] += banked[b];
}

int grid_for(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (int)(g < 1024 ? (g > 0 ? g : 1) : 1024);
}

hj_solver_opts round_opts(const hj_solver_opts& o, const hj_retry_policy& pol, int r) {
  hj_solver_opts q = o;
  const double prod = pol.step_product > 0.0 ? pol.step_product : o.sigma * o.tau;
  q.sigma = o.sigma + r * pol.sigma_step;
  q.tau = prod / q.sigma;
  if (!pol.warm) q.seed = o.seed + (uint64_t)r;
  if (r == pol.rounds && pol.value_tol > 0.0) q.value_tol = pol.value_tol;   // the last round
  return q;
}

template <typename T>
hj_status run_rounds(hj_problem_s* prob, int64_t B, int32_t N, const hj_solver_opts& o,
                     const hj_retry_policy& pol, const double* xq, const double* t, double* V,
                     int32_t* iters, int8_t* status, int8_t* rounds, T* traj_x, T* traj_p,
                     cudaStream_t s) {
  const size_t traj_n = (size_t)B * (size_t)(N + 1) * (size_t)prob->d;
  // workspace: idx [B] | banked [B] | count | (trajectories and warm copies)
  const bool own_traj = pol.warm && (traj_x == nullptr || traj_p == nullptr);
  const size_t head = ((2 * (size_t)B + 1) * sizeof(int32_t) + 255) & ~size_t(255);
  const size_t tbytes = traj_n * sizeof(T);
  const size_t bytes = head + (pol.warm ? 2 * tbytes : 0) + (own_traj ? 2 * tbytes : 0);
  unsigned char* ws = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&ws), bytes, s) != cudaSuccess) return HJ_ERR_OOM;
  int32_t* idx = reinterpret_cast<int32_t*>(ws);
  int32_t* banked = idx + B;
  int32_t* count = banked + B;
  T* wx = pol.warm ? reinterpret_cast<T*>(ws + head) : nullptr;
  T* wp = pol.warm ? wx + traj_n : nullptr;
  if (own_traj) {
    traj_x = reinterpret_cast<T*>(ws + head + 2 * tbytes);
    traj_p = traj_x + traj_n;
  }
  hj_status r = HJ_OK;
  const hj::WarpConfig cfg = shape_for(prob, o.precision, N);
  r = run_solve<T>(prob, B, N, o, cfg, xq, t, V, iters, status, traj_x, traj_p, nullptr, nullptr, s);
  if (r == HJ_OK && cudaMemsetAsync(banked, 0, B * sizeof(int32_t), s) != cudaSuccess) r = HJ_ERR_CUDA;
  if (r == HJ_OK && rounds != nullptr && cudaMemsetAsync(rounds, 0, B, s) != cudaSuccess)
    r = HJ_ERR_CUDA;
  for (int rd = 1; r == HJ_OK && rd <= pol.rounds; ++rd) {
    if (cudaMemsetAsync(count, 0, sizeof(int32_t), s) != cudaSuccess) { r = HJ_ERR_CUDA; break; }
    collect_capped<<<grid_for(B), 256, 0, s>>>(status, iters, B, idx, count, banked);
    int32_t n = 0;
    if (cudaMemcpyAsync(&n, count, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) { r = HJ_ERR_CUDA; break; }
    if (n == 0) break;
    if (pol.warm && (cudaMemcpyAsync(wx, traj_x, tbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
                     cudaMemcpyAsync(wp, traj_p, tbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)) {
      r = HJ_ERR_CUDA;
      break;
    }
    const hj_solver_opts q = round_opts(o, pol, rd);
    hj::SolveArgs<T> a = make_args<T>(prob, n, N, q, xq, t, V, iters, status, traj_x, traj_p,
                                      wx, wp);
    a.idx = idx;
    if (cudaMemsetAsync(prob->counter, 0, hj::kCounterWords * sizeof(unsigned long long), s) !=
        cudaSuccess) {
      r = HJ_ERR_CUDA;
      break;
    }
    r = dispatch<T>(prob, a, cfg, s);
    if (r == HJ_OK && rounds != nullptr) mark_round<<<grid_for(n), 256, 0, s>>>(idx, n, rounds, (int8_t)rd);
  }
  if (r == HJ_OK) add_banked<<<grid_for(B), 256, 0, s>>>(B, iters, banked);
  if (r == HJ_OK && cudaGetLastError() != cudaSuccess) r = HJ_ERR_CUDA;
  if (cudaFreeAsync(ws, s) != cudaSuccess && r == HJ_OK) r = HJ_ERR_CUDA;
  return r;
}

}  // namespace

extern "C" {

hj_status hj_solve_batch_retry(hj_problem prob, int64_t B, const double* xq, const double* t,
                               int32_t N, const hj_solver_opts* opts, const hj_retry_policy* policy,
                               double* V, int32_t* iters, int8_t* status, int8_t* rounds,
                               void* traj_x, void* traj_p, void* stream) {
  if (prob == nullptr || opts == nullptr || policy == nullptr || B < 0) return HJ_ERR_INVALID_ARG;
  if (B > INT32_MAX) return HJ_ERR_INVALID_ARG;   // the retry list holds 32-bit point indices
  if (N < 1 || N > hj::kMaxN) return HJ_ERR_INVALID_ARG;
  const hj_retry_policy& pol = *policy;
  if (pol.rounds < 0 || pol.rounds > 127 || !std::isfinite(pol.sigma_step) ||
      !(pol.step_product >= 0.0) || !std::isfinite(pol.step_product) ||
      !(pol.value_tol >= 0.0) || !std::isfinite(pol.value_tol) ||
      (pol.warm != 0 && pol.warm != 1))
    return HJ_ERR_INVALID_ARG;
  const hj_solver_opts& o = *opts;
  // every round's options must be valid before anything runs
  for (int r = 0; r <= pol.rounds; ++r) {
    const hj_solver_opts q = r == 0 ? o : round_opts(o, pol, r);
    const hj_status oc = check_opts(q);
    if (oc != HJ_OK) return oc;
    const hj_status fc = check_formulation(prob, q);
    if (fc != HJ_OK) return fc;
  }
  if (o.point_offset + B > (int64_t(1) << 32)) return HJ_ERR_INVALID_ARG;
  if (B == 0) return HJ_OK;
  if (xq == nullptr || t == nullptr || V == nullptr || iters == nullptr || status == nullptr)
    return HJ_ERR_INVALID_ARG;
  if ((traj_x == nullptr) != (traj_p == nullptr)) return HJ_ERR_INVALID_ARG;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return HJ_ERR_CUDA;
  if (cur != prob->device) return HJ_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (o.precision == HJ_PREC_FP32)
    return run_rounds<float>(prob, B, N, o, pol, xq, t, V, iters, status, rounds,
                             static_cast<float*>(traj_x), static_cast<float*>(traj_p), s);
  return run_rounds<double>(prob, B, N, o, pol, xq, t, V, iters, status, rounds,
                            static_cast<double*>(traj_x), static_cast<double*>(traj_p), s);
}

}  // extern "C"
