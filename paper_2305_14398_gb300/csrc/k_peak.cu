// Measured FP32 FMA peak of the device (sm_103a): the denominator of the
// ALU-bound roofline fractions (the gate arithmetic of the fused step kernels
// and of the full-state-vector passes is FP32 FMA work).
//
// Every thread runs kChains independent FMA chains x <- x * m + a (m < 1,
// so the values stay bounded and normal), `iters` times; the grid fills every
// SM with kPeakBlocksPerSm blocks.  flops = 2 * kChains * iters * threads.
#include "../../include/tqs.h"
#include "tqs_internal.h"

namespace tqs {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 8;

__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(int iters, float* sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0f + 0.001f * static_cast<float>(threadIdx.x + c);
  const float m = 0.99990f, a = 0.00011f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], m, a);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.0f) sink[threadIdx.x] = s;  // never true: keeps the chains live
}

}  // namespace
}  // namespace tqs

extern "C" tqs_status tqs_measure_fp32_peak(int iters, double* h_tflops, double* h_ms, void* stream) {
  using namespace tqs;
  if (iters < 1 || !h_tflops) {
    set_last_error("tqs_measure_fp32_peak: iters < 1 or h_tflops NULL");
    return TQS_ERR_ARG;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    set_last_error("tqs_measure_fp32_peak: no device");
    return TQS_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = sms * kPeakBlocksPerSm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    set_last_error("tqs_measure_fp32_peak: event");
    return TQS_ERR_CUDA;
  }
  fma_peak_kernel<<<blocks, kPeakThreads, 0, s>>>(iters, nullptr);  // warm
  cudaEventRecord(e0, s);
  fma_peak_kernel<<<blocks, kPeakThreads, 0, s>>>(iters, nullptr);
  cudaEventRecord(e1, s);
  count_launches(2);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || ms <= 0.f) {
    set_last_error("tqs_measure_fp32_peak: kernel failed");
    return TQS_ERR_CUDA;
  }
  const double flops = 2.0 * kChains * 16.0 * iters * double(blocks) * kPeakThreads;
  *h_tflops = flops / (ms * 1e-3) / 1e12;
  if (h_ms) *h_ms = ms;
  return TQS_OK;
}
