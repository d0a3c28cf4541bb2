// Ragged batches: points with their own problem (family, d) and number of time
// steps N, solved by one CUDA-graph launch.
//
// A plan sorts the points into buckets of (problem, N class) with N classes
// 1-32, 33-64, 65-128, 129-256, each bucket's points ordered by decreasing N.
// Each bucket runs one persistent kernel (the
// register-resident kernel with the bucket's launch shape, or the shared-memory
// kernel) that draws the bucket's point ids from its own work counter and
// reads each point's N, xq offset and trajectory offset from device arrays the
// plan uploaded once.  The bucket launches are captured as parallel branches of
// one graph (fork/join over the plan's side streams, largest bucket first), so
// a solve is one cudaGraphLaunch; the graph is re-captured only when the
// caller's buffers change.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "hj_internal.cuh"
#include "hjpdhg.h"
#include "problem.cuh"

using namespace hj_detail;

namespace {

constexpr int kSideStreams = 4;

struct Bucket {
  int prob = 0;
  int ncap = 0;                 // N class upper bound
  int nmax = 0;                 // largest N present
  double work = 0.0;            // sum over points of N * d (launch order)
  std::vector<int32_t> ids;     // host copy of the point ids
  int32_t* d_ids = nullptr;
  hj::WarpConfig cfg{0, 0};     // {0, 0}: shared-memory kernel
  int inner_steps = 0;          // 0: the plan's option
};

int n_class(int N) {
  if (N <= 32) return 32;
  if (N <= 64) return 64;
  if (N <= 128) return 128;
  return 256;
}

}  // namespace

struct hj_ragged_plan_s {
  int device = 0;
  std::vector<hj_problem_s*> probs;
  int64_t B = 0;
  hj_solver_opts opts{};
  std::vector<int64_t> xq_off, traj_off;      // host, B + 1 entries
  int32_t* d_N = nullptr;
  int64_t* d_xq_off = nullptr;
  int64_t* d_traj_off = nullptr;
  unsigned long long* d_counters = nullptr;
  std::vector<Bucket> buckets;                // sorted by decreasing work
  cudaStream_t cap = nullptr;                 // the graph is captured here
  cudaStream_t side[kSideStreams] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kSideStreams] = {};
  cudaGraphExec_t exec = nullptr;
  const void* bound[7] = {};                  // buffers the graph was captured with
};

namespace {

void plan_release(hj_ragged_plan_s* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  for (auto& b : p->buckets) cudaFree(b.d_ids);
  cudaFree(p->d_N); cudaFree(p->d_xq_off); cudaFree(p->d_traj_off); cudaFree(p->d_counters);
  for (int i = 0; i < kSideStreams; ++i) {
    if (p->side[i]) cudaStreamDestroy(p->side[i]);
    if (p->ev_join[i]) cudaEventDestroy(p->ev_join[i]);
  }
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->cap) cudaStreamDestroy(p->cap);
  delete p;
}

template <typename T>
hj_status launch_bucket(hj_ragged_plan_s* p, size_t bi, hj::WarpConfig cfg, const double* xq,
                        const double* t, double* V, int32_t* iters, int8_t* status,
                        void* traj_x, void* traj_p, cudaStream_t s) {
  Bucket& b = p->buckets[bi];
  hj_problem_s* prob = p->probs[b.prob];
  hj::SolveArgs<T> a = make_args<T>(prob, (int64_t)b.ids.size(), b.nmax, p->opts, xq, t, V, iters,
                                    status, traj_x, traj_p, nullptr, nullptr);
  if (b.inner_steps > 0) a.inner_steps = b.inner_steps;
  a.idx = b.d_ids;
  a.Nv = p->d_N;
  a.xq_off = p->d_xq_off;
  a.traj_off = p->d_traj_off;
  a.counter = p->d_counters + (size_t)bi * hj::kCounterWords;
  return dispatch<T>(prob, a, cfg, s);
}

hj_status launch_bucket_any(hj_ragged_plan_s* p, size_t bi, hj::WarpConfig cfg,
                            const double* xq, const double* t, double* V, int32_t* iters,
                            int8_t* status, void* traj_x, void* traj_p, cudaStream_t s) {
  if (p->opts.precision == HJ_PREC_FP32)
    return launch_bucket<float>(p, bi, cfg, xq, t, V, iters, status, traj_x, traj_p, s);
  return launch_bucket<double>(p, bi, cfg, xq, t, V, iters, status, traj_x, traj_p, s);
}

}  // namespace

extern "C" {

hj_status hj_ragged_plan_create(hj_ragged_plan* out, int32_t n_prob, const hj_problem* probs,
                                int64_t B, const int32_t* prob_of, const int32_t* N_of,
                                const hj_solver_opts* opts) {
  if (out == nullptr) return HJ_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_prob < 1 || probs == nullptr || prob_of == nullptr || N_of == nullptr || opts == nullptr)
    return HJ_ERR_INVALID_ARG;
  if (B < 1 || B > INT32_MAX) return HJ_ERR_INVALID_ARG;
  const hj_status oc = check_opts(*opts);
  if (oc != HJ_OK) return oc;
  if (opts->point_offset + B > (int64_t(1) << 32)) return HJ_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HJ_ERR_CUDA;
  for (int i = 0; i < n_prob; ++i) {
    if (probs[i] == nullptr || probs[i]->device != dev) return HJ_ERR_INVALID_ARG;
    const hj_status fc = check_formulation(probs[i], *opts);
    if (fc != HJ_OK) return fc;
  }
  for (int64_t b = 0; b < B; ++b) {
    if (prob_of[b] < 0 || prob_of[b] >= n_prob) return HJ_ERR_INVALID_ARG;
    if (N_of[b] < 1 || N_of[b] > hj::kMaxN) return HJ_ERR_INVALID_ARG;
  }

  hj_ragged_plan_s* p = new (std::nothrow) hj_ragged_plan_s();
  if (p == nullptr) return HJ_ERR_OOM;
  p->device = dev;
  p->probs.assign(probs, probs + n_prob);
  p->B = B;
  p->opts = *opts;
  p->xq_off.resize(B + 1);
  p->traj_off.resize(B + 1);
  p->xq_off[0] = p->traj_off[0] = 0;
  for (int64_t b = 0; b < B; ++b) {
    const int d = probs[prob_of[b]]->d;
    p->xq_off[b + 1] = p->xq_off[b] + d;
    p->traj_off[b + 1] = p->traj_off[b] + (int64_t)(N_of[b] + 1) * d;
  }
  // buckets of (problem, N class)
  std::vector<int> key_of(B);
  std::vector<std::pair<int, int>> keys;
  for (int64_t b = 0; b < B; ++b) {
    const std::pair<int, int> k{prob_of[b], n_class(N_of[b])};
    auto it = std::find(keys.begin(), keys.end(), k);
    if (it == keys.end()) { keys.push_back(k); it = keys.end() - 1; }
    key_of[b] = (int)(it - keys.begin());
  }
  p->buckets.resize(keys.size());
  for (size_t i = 0; i < keys.size(); ++i) {
    p->buckets[i].prob = keys[i].first;
    p->buckets[i].ncap = keys[i].second;
  }
  for (int64_t b = 0; b < B; ++b) {
    Bucket& k = p->buckets[key_of[b]];
    k.ids.push_back((int32_t)b);
    k.nmax = std::max(k.nmax, (int)N_of[b]);
    k.work += (double)N_of[b] * probs[prob_of[b]]->d;
  }
  // within a bucket the kernel draws ids in order: longest N first, so the
  // bucket's tail holds its shortest points
  for (auto& k : p->buckets)
    std::stable_sort(k.ids.begin(), k.ids.end(),
                     [&](int32_t x, int32_t y) { return N_of[x] > N_of[y]; });
  std::sort(p->buckets.begin(), p->buckets.end(),
            [](const Bucket& x, const Bucket& y) { return x.work > y.work; });
  const bool f64 = opts->precision == HJ_PREC_FP64;
  hj_status r = HJ_OK;
  for (auto& k : p->buckets) {
    const hj_problem_s* pr = probs[k.prob];
    k.cfg = hj::default_warp_config(pr->family, pr->d, k.ncap, f64);
    if (k.cfg.G == 0) {
      // shared-memory kernel: the bucket's largest N must fit its shared memory
      const bool drift = pr->family == HJ_FAMILY_TANH_DRIFT;
      const bool mix = opts->scheme != HJ_SCHEME_BE;
      if (pr->family == HJ_FAMILY_QUADCOPTER || pr->family == HJ_FAMILY_GAME_NORMS)
        r = HJ_ERR_UNSUPPORTED;
      else if (pr->family == HJ_FAMILY_EIKONAL) {
        // the captured graph holds no workspace: the state must fit shared memory
        if ((f64 ? hj::eik_cta_smem_bytes<double>(pr->d, k.nmax)
                 : hj::eik_cta_smem_bytes<float>(pr->d, k.nmax)) == 0)
          r = HJ_ERR_UNSUPPORTED;
      } else if ((f64 ? hj::td_cta_smem_bytes<double>(pr->d, k.nmax, drift, mix)
                    : hj::td_cta_smem_bytes<float>(pr->d, k.nmax, drift, mix)) == 0)
        r = HJ_ERR_UNSUPPORTED;
    }
    if (r == HJ_OK) r = upload(&k.d_ids, k.ids.data(), k.ids.size());
  }
  if (r == HJ_OK) r = upload(&p->d_N, N_of, (size_t)B);
  if (r == HJ_OK) r = upload(&p->d_xq_off, p->xq_off.data(), (size_t)B);
  if (r == HJ_OK) r = upload(&p->d_traj_off, p->traj_off.data(), (size_t)B);
  if (r == HJ_OK && cudaMalloc(reinterpret_cast<void**>(&p->d_counters),
                               p->buckets.size() * hj::kCounterWords *
                                   sizeof(unsigned long long)) != cudaSuccess)
    r = HJ_ERR_OOM;
  for (int i = 0; i < kSideStreams && r == HJ_OK; ++i) {
    if (cudaStreamCreateWithFlags(&p->side[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_join[i], cudaEventDisableTiming) != cudaSuccess)
      r = HJ_ERR_CUDA;
  }
  if (r == HJ_OK && cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess)
    r = HJ_ERR_CUDA;
  if (r == HJ_OK && cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess)
    r = HJ_ERR_CUDA;
  if (r != HJ_OK) { plan_release(p); return r; }
  *out = p;
  return HJ_OK;
}

hj_status hj_ragged_plan_destroy(hj_ragged_plan plan) {
  if (plan == nullptr) return HJ_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(plan->device);
  cudaDeviceSynchronize();
  plan_release(plan);
  cudaSetDevice(cur);
  return HJ_OK;
}

hj_status hj_ragged_plan_layout(hj_ragged_plan plan, int64_t* xq_offsets, int64_t* traj_offsets,
                                int32_t* n_buckets) {
  if (plan == nullptr) return HJ_ERR_INVALID_ARG;
  if (xq_offsets)
    std::memcpy(xq_offsets, plan->xq_off.data(), (plan->B + 1) * sizeof(int64_t));
  if (traj_offsets)
    std::memcpy(traj_offsets, plan->traj_off.data(), (plan->B + 1) * sizeof(int64_t));
  if (n_buckets) *n_buckets = (int32_t)plan->buckets.size();
  return HJ_OK;
}

hj_status hj_ragged_plan_bucket(hj_ragged_plan plan, int32_t i, int32_t* problem, int32_t* n_max,
                                int64_t* n_points, int32_t* warps_per_point,
                                int32_t* nodes_per_lane, int32_t* inner_steps) {
  if (plan == nullptr || i < 0 || i >= (int32_t)plan->buckets.size()) return HJ_ERR_INVALID_ARG;
  const Bucket& b = plan->buckets[i];
  if (problem) *problem = b.prob;
  if (n_max) *n_max = b.nmax;
  if (n_points) *n_points = (int64_t)b.ids.size();
  if (warps_per_point) *warps_per_point = b.cfg.half ? 0 : b.cfg.G;
  if (nodes_per_lane) *nodes_per_lane = b.cfg.NPL;
  if (inner_steps) *inner_steps = b.inner_steps > 0 ? b.inner_steps : plan->opts.inner_steps;
  return HJ_OK;
}

hj_status hj_ragged_solve(hj_ragged_plan plan, const double* xq, const double* t, double* V,
                          int32_t* iters, int8_t* status, void* traj_x, void* traj_p,
                          void* stream) {
  if (plan == nullptr || xq == nullptr || t == nullptr || V == nullptr || iters == nullptr ||
      status == nullptr)
    return HJ_ERR_INVALID_ARG;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return HJ_ERR_CUDA;
  if (cur != plan->device) return HJ_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const void* ptrs[7] = {xq, t, V, iters, status, traj_x, traj_p};
  const bool same = plan->exec != nullptr && std::memcmp(ptrs, plan->bound, sizeof(ptrs)) == 0;
  if (!same) {
    // capture on the plan's own stream (the caller's may be the uncapturable
    // legacy default stream); the graph is then launched on the caller's stream
    if (plan->exec) { cudaGraphExecDestroy(plan->exec); plan->exec = nullptr; }
    cudaStream_t c = plan->cap;
    if (cudaStreamBeginCapture(c, cudaStreamCaptureModeRelaxed) != cudaSuccess) return HJ_ERR_CUDA;
    hj_status r = HJ_OK;
    const size_t nb = plan->buckets.size();
    const int nside = (int)std::min<size_t>(nb, kSideStreams);
    if (cudaMemsetAsync(plan->d_counters, 0, nb * hj::kCounterWords * sizeof(unsigned long long),
                        c) != cudaSuccess ||
        cudaEventRecord(plan->ev_fork, c) != cudaSuccess)
      r = HJ_ERR_CUDA;
    for (int i = 0; i < nside && r == HJ_OK; ++i)
      if (cudaStreamWaitEvent(plan->side[i], plan->ev_fork, 0) != cudaSuccess) r = HJ_ERR_CUDA;
    for (size_t bi = 0; bi < nb && r == HJ_OK; ++bi)
      r = launch_bucket_any(plan, bi, plan->buckets[bi].cfg, xq, t, V, iters, status, traj_x,
                            traj_p, plan->side[bi % nside]);
    for (int i = 0; i < nside; ++i) {
      cudaEventRecord(plan->ev_join[i], plan->side[i]);
      cudaStreamWaitEvent(c, plan->ev_join[i], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(c, &g);
    if (r == HJ_OK && (ce != cudaSuccess || g == nullptr)) r = HJ_ERR_CUDA;
    if (r == HJ_OK && cudaGraphInstantiate(&plan->exec, g, 0) != cudaSuccess) r = HJ_ERR_CUDA;
    if (g) cudaGraphDestroy(g);
    if (r != HJ_OK) { plan->exec = nullptr; return r; }
    std::memcpy(plan->bound, ptrs, sizeof(ptrs));
  }
  return cudaGraphLaunch(plan->exec, s) == cudaSuccess ? HJ_OK : HJ_ERR_CUDA;
}

hj_status hj_ragged_autotune(hj_ragged_plan plan, const double* xq, const double* t,
                             int32_t repeats, int32_t max_inner_steps, void* stream) {
  if (plan == nullptr || xq == nullptr || t == nullptr || repeats < 1) return HJ_ERR_INVALID_ARG;
  if (max_inner_steps < 1 || max_inner_steps > 8) return HJ_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool f64 = plan->opts.precision == HJ_PREC_FP64;
  double* V = nullptr;
  int32_t* it = nullptr;
  int8_t* st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hj_status r = HJ_OK;
  if (cudaMalloc(&V, plan->B * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&it, plan->B * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&st, plan->B * sizeof(int8_t)) != cudaSuccess)
    r = HJ_ERR_OOM;
  if (r == HJ_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    r = HJ_ERR_CUDA;
  const int Gs[5] = {0, 1, 2, 4, 8};             // 0: half a warp
  for (size_t bi = 0; bi < plan->buckets.size() && r == HJ_OK; ++bi) {
    Bucket& b = plan->buckets[bi];
    const hj_problem_s* pr = plan->probs[b.prob];
    if (b.cfg.G == 0) continue;                       // shared-memory kernel: nothing to tune
    float best = -1.0f;
    hj::WarpConfig best_c = b.cfg;
    int best_inner = plan->opts.inner_steps;
    // inner gradient steps per x-update: only when the caller allows more than
    // one (they change the iterates, not the fixed point) and H depends on x
    const int inner_hi = (pr->family == HJ_FAMILY_QUADRATIC) ? plan->opts.inner_steps
                         : (max_inner_steps > 1 ? max_inner_steps : plan->opts.inner_steps);
    const int inner_lo = (max_inner_steps > 1 && pr->family != HJ_FAMILY_QUADRATIC)
                         ? 1 : plan->opts.inner_steps;
    for (int inner = inner_lo; inner <= inner_hi && r == HJ_OK; ++inner)
    for (int npl = 1; npl <= 2 && r == HJ_OK; ++npl) {
      for (int gi = 0; gi < 5 && r == HJ_OK; ++gi) {
        const hj::WarpConfig c = Gs[gi] == 0 ? hj::WarpConfig{1, npl, 1} : hj::WarpConfig{Gs[gi], npl};
        if (!hj::warp_config_available(pr->family, pr->d, c, f64) ||
            b.nmax > hj::warp_config_lanes(c) * c.NPL)
          continue;
        b.inner_steps = inner;
        float tot = 0.0f;
        for (int rep = 0; rep <= repeats && r == HJ_OK; ++rep) {
          if (cudaMemsetAsync(plan->d_counters + (size_t)bi * hj::kCounterWords, 0,
                              hj::kCounterWords * sizeof(unsigned long long), s) !=
                  cudaSuccess ||
              cudaEventRecord(e0, s) != cudaSuccess) {
            r = HJ_ERR_CUDA;
            break;
          }
          r = launch_bucket_any(plan, bi, c, xq, t, V, it, st, nullptr, nullptr, s);
          if (r != HJ_OK) break;
          if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            r = HJ_ERR_CUDA;
            break;
          }
          float ms = 0.0f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) tot += ms;
        }
        if (r == HJ_OK && (best < 0.0f || tot < best)) { best = tot; best_c = c; best_inner = inner; }
      }
    }
    b.cfg = best_c;
    b.inner_steps = best_inner;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(V); cudaFree(it); cudaFree(st);
  if (plan->exec) { cudaGraphExecDestroy(plan->exec); plan->exec = nullptr; }
  return r;
}

}  // extern "C"
