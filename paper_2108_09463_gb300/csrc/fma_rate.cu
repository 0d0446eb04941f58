// The device's FP32 fused multiply-add rate, measured: the denominator of the
// roofline of the FP32 micro kernels, which are bound by FP32 and shared-memory
// instruction issue rather than by memory bandwidth. A grid that fills every SM
// runs eight independent FMA chains per thread, either as scalar FP32 FMAs or as
// the paired FP32x2 FMAs (two lanes per instruction) that the micro kernels use,
// and the rate is the FMAs executed (2 flops each) over the kernel's device time.
#include <cuda_runtime.h>

#include "../../include/hmm.h"
#include "hmm_internal.cuh"

namespace hmm {

void set_null_handle_error(const char* msg);

namespace {

constexpr int kRateThreads = 256;
constexpr int kRateChains = 8;

// x <- x b + c on kRateChains independent chains per thread, `iters` times. The
// values stay bounded (b < 1) and the result feeds a comparison, so nothing folds.
template <bool PACKED>
__global__ void __launch_bounds__(kRateThreads) fma_rate_kernel(float b, float c, int iters, float* sink) {
  const float s = 1e-3f * (float)(threadIdx.x + blockIdx.x * blockDim.x);
  float t = 0.f;
  if constexpr (PACKED) {
    float2 x[kRateChains];
#pragma unroll
    for (int k = 0; k < kRateChains; ++k) x[k] = make_float2(s + (float)k, s - (float)k);
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll 8
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int k = 0; k < kRateChains; ++k) x[k] = __ffma2_rn(x[k], b2, c2);
#pragma unroll
    for (int k = 0; k < kRateChains; ++k) t += x[k].x + x[k].y;
  } else {
    float x[kRateChains];
#pragma unroll
    for (int k = 0; k < kRateChains; ++k) x[k] = s + (float)k;
#pragma unroll 8
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int k = 0; k < kRateChains; ++k) x[k] = fmaf(x[k], b, c);
#pragma unroll
    for (int k = 0; k < kRateChains; ++k) t += x[k];
  }
  if (t == -1.0f) *sink = t;   // never true: keeps the chains live
}

}  // namespace
}  // namespace hmm

extern "C" hmm_status hmm_fp32_fma_rate(int packed, double* flops_per_s) {
  using namespace hmm;
  if (!flops_per_s || (packed != 0 && packed != 1)) {
    set_null_handle_error("hmm_fp32_fma_rate: null output or packed not 0/1");
    return HMM_ERR_INVALID_ARG;
  }
  int dev = 0, nsm = 0, per_sm = 0;
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t st = nullptr;
  hmm_status s = HMM_ERR_CUDA;
  float ms = 0.f;
  const int iters = 1 << 16;
  auto kern = packed ? fma_rate_kernel<true> : fma_rate_kernel<false>;
  do {
    if (cudaGetDevice(&dev) != cudaSuccess) break;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) break;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRateThreads, 0) != cudaSuccess || per_sm < 1)
      break;
    if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) {
      s = HMM_ERR_OUT_OF_MEMORY;
      break;
    }
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) break;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) break;
    const int grid = per_sm * nsm;
    kern<<<grid, kRateThreads, 0, st>>>(0.999999f, 1e-7f, iters / 16, sink);   // warm-up
    if (cudaEventRecord(e0, st) != cudaSuccess) break;
    kern<<<grid, kRateThreads, 0, st>>>(0.999999f, 1e-7f, iters, sink);
    if (cudaEventRecord(e1, st) != cudaSuccess) break;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) break;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)) break;
    const double fmas = (double)grid * kRateThreads * (double)iters * kRateChains * (packed ? 2.0 : 1.0);
    *flops_per_s = 2.0 * fmas / (ms * 1e-3);
    s = HMM_OK;
  } while (false);
  if (s == HMM_ERR_OUT_OF_MEMORY) set_null_handle_error("hmm_fp32_fma_rate: cudaMalloc of the result word failed");
  else if (s != HMM_OK) set_null_handle_error("hmm_fp32_fma_rate: CUDA call failed");
  else set_null_handle_error("");
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (sink) cudaFree(sink);
  return s;
}
