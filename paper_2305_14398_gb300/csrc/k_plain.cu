// Plain materialised form (sm_103a): stage 4 (Algorithm 2, the step unitary
// written out as a dense matrix) and stage 6 applied per step (eq. 11, dense
// matrix-vector product).  This is the baseline the fused kernel is measured
// against; both kernels stream the 2^n x 2^n complex64 matrix through HBM.
#include "checked.h"
#include "step_entry.h"
#include "tqs_internal.h"

namespace tqs {
namespace {

// S[r][c] = prod_f M_f[bits_f(r)][bits_f(c)] when r and c agree on every idle
// qubit (identity factors), else 0 (step_entry.h).  Factors are staged in
// shared memory.
constexpr int kMatThreads = 256;
constexpr int kMaxFactors = 16;

__global__ void __launch_bounds__(kMatThreads)
    materialize_kernel(const StepFactor* __restrict__ factors, int nf, uint32_t idle, int n,
                       float2* __restrict__ S) {
  __shared__ StepFactor fs[kMaxFactors];
  for (int i = threadIdx.x; i < nf * static_cast<int>(sizeof(StepFactor) / 8); i += blockDim.x)
    reinterpret_cast<float2*>(fs)[TQS_IX(i, int(sizeof(fs) / 8))] =
        reinterpret_cast<const float2*>(factors)[i];
  __syncthreads();
  const int64_t N = int64_t(1) << n;
  const int64_t pairs = (N * N) >> 1;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < pairs; e += stride) {
    const int64_t flat = e << 1;
    const uint32_t r = static_cast<uint32_t>(flat >> n);
    const uint32_t c = static_cast<uint32_t>(flat & (N - 1));
    const float2 v0 = step_entry(fs, nf, idle, r, c);
    const float2 v1 = step_entry(fs, nf, idle, r, c + 1);
    __stcs(reinterpret_cast<float4*>(S) + TQS_IX(e, pairs), make_float4(v0.x, v0.y, v1.x, v1.y));
  }
}

// y = S x: one warp per row, float4 (two amplitudes) per lane per iteration.
constexpr int kMvWarps = 8;

__global__ void __launch_bounds__(kMvWarps * 32)
    matvec_kernel(const float2* __restrict__ S, const float2* __restrict__ x,
                  float2* __restrict__ y, int n) {
  const int64_t N = int64_t(1) << n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row = int64_t(blockIdx.x) * kMvWarps + warp;
  if (row >= N) return;
  const float4* srow = reinterpret_cast<const float4*>(S) + TQS_IX(row, N) * (N >> 1);
  const float4* x4 = reinterpret_cast<const float4*>(x);
  float re = 0.f, im = 0.f;
  for (int64_t k = lane; k < (N >> 1); k += 32) {
    const float4 s = __ldcs(srow + TQS_IX(k, N >> 1));
    const float4 v = __ldg(x4 + TQS_IX(k, N >> 1));
    re = fmaf(s.x, v.x, re);
    re = fmaf(-s.y, v.y, re);
    re = fmaf(s.z, v.z, re);
    re = fmaf(-s.w, v.w, re);
    im = fmaf(s.x, v.y, im);
    im = fmaf(s.y, v.x, im);
    im = fmaf(s.z, v.w, im);
    im = fmaf(s.w, v.z, im);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) y[row] = make_float2(re, im);
}

}  // namespace

TQS_DEFINE_VIOLATIONS(violations_plain)

namespace {

int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

}  // namespace

cudaError_t launch_materialize(const StepFactor* d_factors, StepDesc step, int n, float2* d_S,
                               cudaStream_t s) {
  if (step.f_count > kMaxFactors) return cudaErrorInvalidValue;
  const int64_t N = int64_t(1) << n;
  const int64_t pairs = (N * N) >> 1;
  int64_t blocks = (pairs + kMatThreads - 1) / kMatThreads;
  const int64_t cap = int64_t(sm_count()) * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  materialize_kernel<<<static_cast<int>(blocks), kMatThreads, 0, s>>>(
      d_factors + step.f_begin, step.f_count, step.idle, n, d_S);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_matvec(const float2* d_S, const float2* d_x, float2* d_y, int n,
                          cudaStream_t s) {
  const int64_t N = int64_t(1) << n;
  const int64_t blocks = (N + kMvWarps - 1) / kMvWarps;
  matvec_kernel<<<static_cast<int>(blocks), kMvWarps * 32, 0, s>>>(d_S, d_x, d_y, n);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace tqs
