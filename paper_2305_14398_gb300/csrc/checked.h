// Bounds checks of the TQS_CHECKED build.
//
// In that build every global and shared-memory index a kernel computes goes
// through TQS_IX(i, n): an index outside [0, n) is counted in this
// translation unit's device counter and replaced by 0, so the access stays in
// bounds (no fault, no trap) and a test can run the kernels and require the
// count to stay 0.  In the normal build TQS_IX(i, n) is i.
//
// Each .cu file includes this header once and defines its host accessor with
// TQS_DEFINE_VIOLATIONS(name); check_violations() in k_fused.cu sums them.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#ifdef TQS_CHECKED
namespace tqs {
namespace {
__device__ unsigned int g_tu_violations;

template <class I, class N>
__device__ __forceinline__ I checked_index(I i, N n) {
  if (static_cast<unsigned long long>(static_cast<long long>(i)) >=
      static_cast<unsigned long long>(n)) {
    atomicAdd(&g_tu_violations, 1u);
    return I(0);
  }
  return i;
}
}  // namespace
}  // namespace tqs
#define TQS_IX(i, n) ::tqs::checked_index((i), (n))
#define TQS_DEFINE_VIOLATIONS(name)                                                    \
  cudaError_t name(unsigned int* count, bool reset) {                                  \
    cudaError_t e = cudaMemcpyFromSymbol(count, g_tu_violations, sizeof(unsigned int)); \
    if (e == cudaSuccess && reset) {                                                   \
      const unsigned int zero = 0;                                                     \
      e = cudaMemcpyToSymbol(g_tu_violations, &zero, sizeof(zero));                    \
    }                                                                                  \
    return e;                                                                          \
  }
#else
#define TQS_IX(i, n) ((void)(n), (i))
#define TQS_DEFINE_VIOLATIONS(name)                   \
  cudaError_t name(unsigned int* count, bool reset) { \
    (void)reset;                                      \
    *count = 0;                                       \
    return cudaSuccess;                               \
  }
#endif
