// Probabilities and their FP64 sum (sm_103a).
//
// p_i = |psi_i|^2 (Sec. 2.1, eq. 2) correctly rounded to FP64 from the FP32
// parts (their squares are exact FP64 values, built with integer operations:
// GB300 runs FP64 arithmetic at about 1/64 of its FP32 rate, so each
// probability costs one FP64 add instead of two widenings, a multiply and a
// fused multiply-add), optionally written out, and summed over the
// indices i with (i & zero_mask) == 0 (zero_mask = 0: the norm; otherwise the
// marginal probability that the masked qubits read 0, as for the
// Deutsch-Jozsa input register of Sec. 2.5).  The reduction runs in a fixed
// order: per-block partial sums into scratch, then one warp sums the
// partials, so the result does not depend on scheduling.
#include <mutex>

#include "../../include/tqs.h"
#include "checked.h"
#include "exact_sq.h"
#include "tqs_internal.h"

namespace tqs {
namespace {

constexpr int kProbThreads = 256;
constexpr int64_t kAmpsPerBlock = 8192;
constexpr int kMaxPartials = 1024;

__global__ void __launch_bounds__(kProbThreads)
    probs_kernel(const float2* __restrict__ st, int64_t N, int64_t chunk, double* __restrict__ probs,
                 uint64_t zero_mask, double* __restrict__ partials) {
  const int64_t begin = int64_t(blockIdx.x) * chunk;
  int64_t end = begin + chunk;
  if (end > N) end = N;
  double acc = 0.0;
  for (int64_t i = begin + 2 * threadIdx.x; i < end; i += 2 * kProbThreads) {
    const float4 v = __ldcs(reinterpret_cast<const float4*>(st) + TQS_IX(i >> 1, N >> 1));
    const double q0 = sq_sum_f64(v.x, v.y);
    const double q1 = sq_sum_f64(v.z, v.w);
    if (probs) __stcs(reinterpret_cast<double2*>(probs) + TQS_IX(i >> 1, N >> 1), make_double2(q0, q1));
    if ((static_cast<uint64_t>(i) & zero_mask) == 0) acc += q0;
    if ((static_cast<uint64_t>(i + 1) & zero_mask) == 0) acc += q1;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[kProbThreads / 32];
  if ((threadIdx.x & 31) == 0) red[TQS_IX(threadIdx.x >> 5, kProbThreads / 32)] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kProbThreads / 32; ++w) s += red[w];
    partials[TQS_IX(blockIdx.x, gridDim.x)] = s;
  }
}

__global__ void sum_partials_kernel(const double* __restrict__ partials, int count,
                                    double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += 32) acc += partials[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x == 0) *out = acc;
}

}  // namespace

TQS_DEFINE_VIOLATIONS(violations_probs)

int probs_partial_count(int n) {
  const int64_t N = int64_t(1) << n;
  int64_t blocks = (N + kAmpsPerBlock - 1) / kAmpsPerBlock;
  if (blocks > kMaxPartials) blocks = kMaxPartials;
  if (blocks < 1) blocks = 1;
  return static_cast<int>(blocks);
}

cudaError_t launch_probs(const float2* d_state, int n, double* d_probs, uint64_t zero_mask,
                         double* d_partials, int n_partials, double* d_sum, cudaStream_t s) {
  const int64_t N = int64_t(1) << n;
  int64_t chunk = (N + n_partials - 1) / n_partials;
  chunk = (chunk + 1) & ~int64_t(1);
  probs_kernel<<<n_partials, kProbThreads, 0, s>>>(d_state, N, chunk, d_probs, zero_mask,
                                                   d_partials);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || d_sum == nullptr) return e;
  sum_partials_kernel<<<1, 32, 0, s>>>(d_partials, n_partials, d_sum);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free variant (tqs_probabilities_noalloc).
//
// Its per-block partial sums live in this fixed array, loaded with the library
// and kept by every GPU that loads it until the process exits.  Host code may
// not use the array's name as a device address: the address is looked up with
// cudaGetSymbolAddress once per device, with that device current, and cached.
// Each call overwrites all the partials it reads, so nothing needs clearing
// between calls; calls that overlap on the GPU share the array and race.  The
// cached address belongs to the device's primary context (the one the CUDA
// runtime uses): it is not valid after cudaDeviceReset or in another context
// made current on the same device.
// ---------------------------------------------------------------------------
constexpr int kStaticPartials = kMaxPartials;  // 1024 doubles = 8 KiB
static __device__ __align__(256) double g_static_partials[kStaticPartials];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
double* g_static_ptr[kMaxDevices] = {};
}  // namespace

}  // namespace tqs

extern "C" tqs_status tqs_probabilities_noalloc(const tqs_c64* d_state, int n, double* d_probs,
                                                double* d_sum, void* stream) {
  using namespace tqs;
  if (!d_state) {
    set_last_error("tqs_probabilities_noalloc: d_state is NULL");
    return TQS_ERR_ARG;
  }
  if (n < 1 || n > 30) {
    set_last_error("tqs_probabilities_noalloc: n must be in [1, 30]");
    return TQS_ERR_TOO_MANY_QUBITS;
  }
  if ((reinterpret_cast<uintptr_t>(d_state) & 15u) || (reinterpret_cast<uintptr_t>(d_probs) & 15u)) {
    set_last_error("tqs_probabilities_noalloc: device buffers must be 16-byte aligned");
    return TQS_ERR_ARG;
  }
  // probs_partial_count never exceeds kMaxPartials, which the array holds
  static_assert(kStaticPartials >= kMaxPartials, "the fixed array holds every partial count");
  const int parts = probs_partial_count(n);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_last_error("tqs_probabilities_noalloc: no usable current device");
    return TQS_ERR_CUDA;
  }
  double* partials = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_static_partials);
      if (e != cudaSuccess || ptr == nullptr) {
        set_last_error("tqs_probabilities_noalloc: cudaGetSymbolAddress failed");
        return TQS_ERR_CUDA;
      }
      g_static_ptr[dev] = static_cast<double*>(ptr);
    }
    partials = g_static_ptr[dev];
  }
  e = launch_probs(reinterpret_cast<const float2*>(d_state), n, d_probs, 0, partials, parts, d_sum,
                   static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    set_last_error("tqs_probabilities_noalloc: kernel launch failed");
    return TQS_ERR_CUDA;
  }
  return TQS_OK;
}
