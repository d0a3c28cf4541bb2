// FP32 FMA throughput of the device, measured: the denominator of the roofline
// fraction of the FP32 iteration kernels (which are bound by the FP32 FMA pipe),
// taken on the same GPU and clocks as the kernels instead of derived from the
// SM count and the maximum clock.  Diagnostic only; the method has no
// counterpart.
//
// Every thread runs 8 independent chains v <- v * a + b (scalar fmaf, or the
// packed two-wide form on 4 float2 chains), so the FMA pipe, not latency, bounds
// the launch; the grid fills every SM at full occupancy.
#include <cuda_runtime.h>

#include "hjpdhg.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) fma_chains(float* out, int64_t iters, float a, float b) {
  float v[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) v[i] = 1e-3f * (float)(threadIdx.x + i);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r)
#pragma unroll
      for (int i = 0; i < kChains; ++i) v[i] = fmaf(v[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += v[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) fma2_chains(float* out, int64_t iters, float a, float b) {
  float2 v[kChains / 2];
#pragma unroll
  for (int i = 0; i < kChains / 2; ++i)
    v[i] = make_float2(1e-3f * (float)(threadIdx.x + 2 * i), 1e-3f * (float)(threadIdx.x + 2 * i + 1));
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r)
#pragma unroll
      for (int i = 0; i < kChains / 2; ++i) v[i] = __ffma2_rn(v[i], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains / 2; ++i) s += v[i].x + v[i].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" hj_status hj_probe_fp32_fma(int64_t iters, int32_t packed, double* tflops,
                                       void* stream) {
  if (iters < 1 || tflops == nullptr) return HJ_ERR_INVALID_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HJ_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HJ_ERR_CUDA;
  const int block = 256, grid = nsm * 8;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  float* out = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&out), sizeof(float) * grid * block, s) !=
      cudaSuccess)
    return HJ_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hj_status r = HJ_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) r = HJ_ERR_CUDA;
  float ms = 0.f;
  if (r == HJ_OK) {
    // warm-up launch, then the timed one
    for (int rep = 0; rep < 2 && r == HJ_OK; ++rep) {
      if (rep == 1 && cudaEventRecord(e0, s) != cudaSuccess) r = HJ_ERR_CUDA;
      if (packed)
        fma2_chains<<<grid, block, 0, s>>>(out, iters, 0.999f, 1e-4f);
      else
        fma_chains<<<grid, block, 0, s>>>(out, iters, 0.999f, 1e-4f);
      if (cudaGetLastError() != cudaSuccess) r = HJ_ERR_CUDA;
    }
    if (r == HJ_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                       cudaEventSynchronize(e1) != cudaSuccess ||
                       cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)))
      r = HJ_ERR_CUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && r == HJ_OK) r = HJ_ERR_CUDA;
  if (r != HJ_OK) return r;
  const double fmas = (double)grid * block * kChains * kUnroll * (double)iters;
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return HJ_OK;
}
