// hj_solve_batch_static: the batched solve for callers that must not allocate
// device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory budget
// fixed before it starts (an allocator owned by a host framework, a real-time
// loop that forbids allocation after start-up), or code that only receives
// buffers it did not allocate.  hj_problem_create allocates the problem's
// parameter copies and the persistent kernels' work counter; this entry point
// instead keeps both in one file-scope __device__ array of fixed size, so the
// call allocates nothing.  The kernels and their arithmetic are the ones
// hj_solve_batch runs; only where the parameters and the counter live differs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "hj_internal.cuh"
#include "hjpdhg.h"
#include "problem.cuh"

using namespace hj_detail;

namespace {

// Every GPU that loads the library holds this array until the process exits.
constexpr size_t kStaticScratchBytes = 64 * 1024;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};   // device address of the array, per device

// Host staging of the parameter block (no heap allocation either).
alignas(256) unsigned char g_stage[kStaticScratchBytes];

size_t up256(size_t v) { return (v + 255) & ~size_t(255); }

// Byte layout of the array for (d, tanh-drift A present, iterate size):
// counter | W2 | W | c | A64 | A (iterate type) | A^T (iterate type).
struct StaticLayout {
  size_t counter = 0, W2, W, c, A64, A, At, total;
  StaticLayout(int d, bool has_A, size_t tsize) {
    W2 = 256;
    W = W2 + up256(d * sizeof(double));
    c = W + up256(d * sizeof(double));
    A64 = c + up256(d * sizeof(double));
    const size_t nA = has_A ? (size_t)d * d : 0;
    A = A64 + up256(nA * sizeof(double));
    At = A + up256(nA * tsize);
    total = At + up256(nA * tsize);
  }
};

// Set-up, once per device, with that device current: the address of the
// array as the device sees it (its name in host code is only a stand-in).
hj_status scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return HJ_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> g(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr)
      return HJ_ERR_CUDA;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return HJ_OK;
}

}  // namespace

extern "C" {

int64_t hj_static_scratch_bytes(void) { return (int64_t)kStaticScratchBytes; }

hj_status hj_solve_batch_static(int32_t family, int32_t d, const double* dyn, int64_t n_dyn,
                                const double* W, const double* c, int64_t B, const double* xq,
                                const double* t, int32_t N, const hj_solver_opts* opts,
                                double* V, int32_t* iters, int8_t* status, void* traj_x,
                                void* traj_p, void* stream) {
  // argument checks shared with hj_problem_create / hj_solve_batch
  if (opts == nullptr || W == nullptr || c == nullptr || B < 0) return HJ_ERR_INVALID_ARG;
  if (d < 1 || d > hj::kMaxD || n_dyn < 0 || (n_dyn > 0 && dyn == nullptr))
    return HJ_ERR_INVALID_ARG;
  switch (family) {
    case HJ_FAMILY_QUADRATIC: if (n_dyn != 0) return HJ_ERR_INVALID_ARG; break;
    case HJ_FAMILY_QUADCOPTER:
      if (d != 12 || n_dyn != 4 || !(dyn[0] > 0.0) || !(dyn[3] >= 0.0)) return HJ_ERR_INVALID_ARG;
      break;
    case HJ_FAMILY_TANH_DRIFT: if (n_dyn != (int64_t)d * d) return HJ_ERR_INVALID_ARG; break;
    case HJ_FAMILY_EIKONAL: return HJ_ERR_UNSUPPORTED;   // no bump-centre slot in the array
    case HJ_FAMILY_GAME_NORMS: return HJ_ERR_UNSUPPORTED;
    default: return HJ_ERR_INVALID_ARG;
  }
  if (!all_finite(W, d) || !all_finite(c, d) || (n_dyn > 0 && !all_finite(dyn, n_dyn)))
    return HJ_ERR_INVALID_ARG;
  if (N < 1 || N > hj::kMaxN) return HJ_ERR_INVALID_ARG;
  const hj_status oc = check_opts(*opts);
  if (oc != HJ_OK) return oc;
  // the problem view below, with the host-side facts hj_problem_create records
  // about W, so that the option checks of hj_solve_batch apply unchanged
  hj_problem_s view;
  view.family = family;
  view.d = d;
  view.w_nonzero = true;
  view.w2max = 0.0;
  for (int i = 0; i < d; ++i) {
    if (W[i] == 0.0) view.w_nonzero = false;
    view.w2max = std::max(view.w2max, W[i] * W[i]);
  }
  for (int i = 0; i < 4; ++i) view.qc[i] = (family == HJ_FAMILY_QUADCOPTER) ? dyn[i] : 0.0;
  const hj_status fc = check_formulation(&view, *opts);
  if (fc != HJ_OK) return fc;
  if (opts->point_offset + B > (int64_t(1) << 32)) return HJ_ERR_INVALID_ARG;
  const bool has_A = family == HJ_FAMILY_TANH_DRIFT;
  const size_t tsize = opts->precision == HJ_PREC_FP32 ? sizeof(float) : sizeof(double);
  const StaticLayout L(d, has_A, tsize);
  if (L.total > kStaticScratchBytes) return HJ_ERR_UNSUPPORTED;   // parameters do not fit
  if (B == 0) return HJ_OK;
  if (xq == nullptr || t == nullptr || V == nullptr || iters == nullptr || status == nullptr)
    return HJ_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HJ_ERR_CUDA;
  unsigned char* base = nullptr;
  hj_status r = scratch_address(dev, &base);
  if (r != HJ_OK) return r;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  {
    // stage the parameter block on the host and copy it into the array; the
    // counter starts at zero for every call
    std::lock_guard<std::mutex> g(g_mu);
    std::memset(g_stage, 0, L.total);
    double* w2 = reinterpret_cast<double*>(g_stage + L.W2);
    double* ws = reinterpret_cast<double*>(g_stage + L.W);
    double* cs = reinterpret_cast<double*>(g_stage + L.c);
    for (int i = 0; i < d; ++i) { w2[i] = W[i] * W[i]; ws[i] = W[i]; cs[i] = c[i]; }
    if (has_A) {
      double* a64 = reinterpret_cast<double*>(g_stage + L.A64);
      for (int i = 0; i < d * d; ++i) a64[i] = dyn[i];
      for (int i = 0; i < d; ++i)
        for (int k = 0; k < d; ++k) {
          const double v = dyn[(size_t)i * d + k];
          if (tsize == sizeof(float)) {
            reinterpret_cast<float*>(g_stage + L.A)[(size_t)i * d + k] = (float)v;
            reinterpret_cast<float*>(g_stage + L.At)[(size_t)k * d + i] = (float)v;
          } else {
            reinterpret_cast<double*>(g_stage + L.A)[(size_t)i * d + k] = v;
            reinterpret_cast<double*>(g_stage + L.At)[(size_t)k * d + i] = v;
          }
        }
    }
    // pageable source: the call returns once the bytes are staged for the copy
    if (cudaMemcpyAsync(base, g_stage, L.total, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return HJ_ERR_CUDA;
  }

  // the view's device pointers all point into the array
  view.device = dev;
  view.W2 = reinterpret_cast<double*>(base + L.W2);
  view.W = reinterpret_cast<double*>(base + L.W);
  view.c = reinterpret_cast<double*>(base + L.c);
  view.counter = reinterpret_cast<unsigned long long*>(base + L.counter);
  if (has_A) {
    view.Ad = reinterpret_cast<double*>(base + L.A64);
    if (tsize == sizeof(float)) {
      view.Af = reinterpret_cast<float*>(base + L.A);
      view.Atf = reinterpret_cast<float*>(base + L.At);
    } else {
      view.Atd = reinterpret_cast<double*>(base + L.At);
      // the FP64 kernels read A through Ad; the A64 block holds the same values
    }
  }
  const hj::WarpConfig cfg = shape_for(&view, opts->precision, N);
  if (opts->precision == HJ_PREC_FP32)
    r = run_solve<float>(&view, B, N, *opts, cfg, xq, t, V, iters, status, traj_x, traj_p,
                         nullptr, nullptr, s);
  else
    r = run_solve<double>(&view, B, N, *opts, cfg, xq, t, V, iters, status, traj_x, traj_p,
                          nullptr, nullptr, s);
  return r;   // the view owns nothing; its pointers die with it
}

}  // extern "C"
