// Exact square of an FP32 value as an FP64 bit pattern, with integer
// operations only (GB300's FP64 pipe is ~1/64 of its FP32 rate, so the
// per-amplitude |psi|^2 avoids it except for one correctly rounded add).
//
// x = m * 2^(e - 150) with a 24-bit integer significand m (after normalising
// subnormals); x^2 = m^2 * 2^(2e - 300) where m^2 < 2^48 fits an FP64
// significand exactly.  The result is bit-identical to (double)x * (double)x.
// Host and device code (the host build is the unit test's).
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define TQS_HD __host__ __device__ __forceinline__
#else
#define TQS_HD inline
#endif

namespace tqs {

TQS_HD int clz32(uint32_t v) {
#if defined(__CUDA_ARCH__)
  return __clz(static_cast<int>(v));
#else
  return v ? __builtin_clz(v) : 32;
#endif
}

TQS_HD uint64_t sq_f32_as_f64_bits_general(uint32_t xbits);

// Normal x (the common case): m in [2^23, 2^24), m^2 in [2^46, 2^48).  The
// significand field is m^2 shifted so that its leading one lands on bit 52;
// adding the exponent field one below the biased exponent absorbs that
// leading one, so no mask is needed.
TQS_HD uint64_t sq_f32_as_f64_bits(uint32_t xbits) {
  const uint32_t a = xbits & 0x7fffffffu;
  if (a < 0x00800000u) return sq_f32_as_f64_bits_general(xbits);  // zero or subnormal
  const uint32_t m = (a & 0x7fffffu) | 0x800000u;
  const int e = static_cast<int>(a >> 23);
  const uint64_t X = static_cast<uint64_t>(m) * m;
  const bool top47 = (static_cast<uint32_t>(X >> 32) >> 15) != 0;  // bit 47 of X
  const uint64_t Y = X << (top47 ? 5 : 6);
  // biased exponent 2e - 254 + 1023 (top bit 47) or one less (top bit 46), minus 1
  const uint64_t ebits = static_cast<uint64_t>(2 * e + 768 + (top47 ? 1 : 0)) << 52;
  return ebits + Y;
}

// Any finite x, subnormals included.
TQS_HD uint64_t sq_f32_as_f64_bits_general(uint32_t xbits) {
  const uint32_t a = xbits & 0x7fffffffu;
  int e = static_cast<int>(a >> 23);
  uint32_t m = a & 0x7fffffu;
  if (e == 0) {
    if (m == 0) return 0;
    const int s = clz32(m) - 8;  // bring the leading one to bit 23
    m <<= s;
    e = 1 - s;
  } else {
    m |= 0x800000u;
  }
  const uint64_t X = static_cast<uint64_t>(m) * m;  // in [2^46, 2^48)
  const int top = (X >> 47) ? 47 : 46;
  const int E = top + 2 * e - 300;                   // unbiased FP64 exponent
  const uint64_t frac = (X << (52 - top)) & ((uint64_t(1) << 52) - 1);
  return (static_cast<uint64_t>(E + 1023) << 52) | frac;
}

#if defined(__CUDACC__)
// |x + iy|^2 correctly rounded to FP64 (bit-identical to (double)x * x +
// (double)y * y): the two squares are exact FP64 values built with integer
// operations, one FP64 add rounds their sum.
__device__ __forceinline__ double sq_sum_f64(float x, float y) {
  const double a = __longlong_as_double(static_cast<long long>(sq_f32_as_f64_bits(__float_as_uint(x))));
  const double b = __longlong_as_double(static_cast<long long>(sq_f32_as_f64_bits(__float_as_uint(y))));
  return __dadd_rn(a, b);
}
#endif

}  // namespace tqs
