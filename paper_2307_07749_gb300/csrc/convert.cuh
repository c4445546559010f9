// convert.cuh - FP64 <-> FP32 conversions on the integer pipes.
//
// On GB300 the FP64 pipe runs at 1/64 of the FP32 rate and the hardware FP64<->FP32 conversions
// occupy it, so kernels that compute in FP32 (or double-float) but read and write FP64 vectors
// convert with integer bit operations instead.  Both functions are exact IEEE conversions for
// normal numbers; magnitudes below 2^-126 flush to signed zero.
#pragma once
#include <stdint.h>
#include <string.h>

namespace bltt {

#if defined(__CUDACC__)
#define BLTT_HD __host__ __device__ __forceinline__
#else
#define BLTT_HD inline
#endif

BLTT_HD uint64_t bits_d(double x) { uint64_t b; memcpy(&b, &x, 8); return b; }
BLTT_HD double from_bits_d(uint64_t b) { double x; memcpy(&x, &b, 8); return x; }
BLTT_HD uint32_t bits_f(float x) { uint32_t b; memcpy(&b, &x, 4); return b; }
BLTT_HD float from_bits_f(uint32_t b) { float x; memcpy(&x, &b, 4); return x; }

// double -> float, round to nearest even; |x| >= 2^128 (and Inf/NaN) -> +-Inf
BLTT_HD float d2f_bits(double x) {
  const uint64_t b = bits_d(x);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  const uint32_t m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);      // top 23 mantissa bits
  const uint32_t rest = lo & 0x1FFFFFFFu;                       // 29 dropped bits
  const uint32_t up = (rest > 0x10000000u) | ((rest == 0x10000000u) & (m & 1u));
  uint32_t f = ((uint32_t)e << 23) + m + up;                    // a carry moves into the exponent
  if (e <= 0) f = 0u;
  if (e >= 255) f = 0x7F800000u;
  return from_bits_f(f | sign);
}

// float -> double (exact); zeros and subnormals -> signed zero, Inf/NaN kept
BLTT_HD double f2d_bits(float x) {
  const uint32_t b = bits_f(x);
  const uint32_t sign = b & 0x80000000u;
  const uint32_t e = (b >> 23) & 0xFFu;
  const uint32_t m = b & 0x7FFFFFu;
  uint32_t hi = sign | ((e + 896u) << 20) | (m >> 3);
  if (e == 0u) hi = sign;
  if (e == 255u) hi = sign | 0x7FF00000u | (m >> 3);
  const uint32_t lo = (e == 0u) ? 0u : (m << 29);
  return from_bits_d(((uint64_t)hi << 32) | lo);
}

// Cheaper conversions for the FP32 kernels, whose values only need FP32 accuracy on the way in
// and exactness on the way out.
//
// double -> float rounded to nearest with ties away from zero (ties to even differs only on
// exact ties, by one ulp); magnitudes below 2^-126 flush to signed zero; |x| >= 2^128, Inf and
// NaN become NaN (so that a breakdown stays visible).
BLTT_HD float d2f_fast(double x) {
  const uint64_t b = bits_d(x);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t sign = hi & 0x80000000u, e = hi & 0x7FF00000u;
  const uint32_t t = hi - 0x38000000u;                 // exponent - (1023 - 127), in place
  uint32_t f = ((t << 3) | (lo >> 29)) & 0x7FFFFFFFu;  // exponent and top 23 mantissa bits
  f += (lo >> 28) & 1u;                                // the first dropped bit rounds
  f |= sign;
  if (e < 0x38100000u) f = sign;                       // below 2^-126
  if (e >= 0x47F00000u) f = 0x7FC00000u | sign;        // 2^128 and beyond, Inf, NaN
  return from_bits_f(f);
}

// float -> double, exact for normal numbers and zeros; Inf and NaN become NaN; subnormal inputs
// (below 2^-126) are not exact
BLTT_HD double f2d_fast(float x) {
  const uint32_t b = bits_f(x);
  const uint32_t a = b & 0x7FFFFFFFu, sign = b & 0x80000000u;
  uint32_t hi = ((a >> 3) + 0x38000000u) | sign;
  if (a == 0u) hi = sign;
  if (a >= 0x7F800000u) hi = 0x7FF80000u | sign;
  return from_bits_d(((uint64_t)hi << 32) | (uint32_t)(b << 29));
}

}  // namespace bltt
