// Split of an FP64 value into two BF16 values, x ~ hi + lo with hi = bf16(x) and
// lo = bf16(x - hi) (round to nearest, ties to even), taken from the IEEE-754
// bit patterns with integer arithmetic only.  The BF16x2 sigma splits FP64 vectors
// this way before every product; on this GPU FP64 conversions run on the narrow
// FP64 pipe, integer operations on the full-rate ALUs.
//
// BF16 keeps 8 significant bits and the binary32 exponent range.  bf16_split_bits
// handles every finite x whose hi and lo are zero or normal BF16 numbers (|x| in
// [2^-126, 2^127] and x - hi either 0 or at least 2^-126 in magnitude) and returns
// false otherwise (subnormal or overflowing parts, infinities, NaN); callers use a
// conversion routine for those.  Host-compilable so that it can be checked against
// exact rational arithmetic on the CPU.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define FORTE_HD __host__ __device__ __forceinline__
#else
#define FORTE_HD inline
#endif

namespace forte {

FORTE_HD uint64_t f64_bits(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}

FORTE_HD int clz64(uint64_t v) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)v);
#else
  return __builtin_clzll(v);
#endif
}

// |x| = m 2^(E - 52) with m = 2^52 + mantissa (normal x): hi keeps the top 8 bits of
// m rounded to nearest-even, and the remainder d = m - m_hi (|d| <= 2^44, in units
// of 2^(E - 52)) is rounded the same way for lo.
FORTE_HD bool bf16_split_bits(double x, uint16_t &hi, uint16_t &lo) {
  const uint64_t b = f64_bits(x);
  const uint32_t sign = (uint32_t)(b >> 63);
  const int e = (int)((b >> 52) & 0x7FF);  // biased FP64 exponent
  const uint64_t frac = b & ((1ull << 52) - 1);
  if (e == 0 && frac == 0) {  // +-0: both parts are the signed zero / +0
    hi = (uint16_t)(sign << 15);
    lo = 0;
    return true;
  }
  const int E = e - 1023;  // unbiased exponent of x
  if (e == 0 || E < -126 || E > 127) return false;
  // hi: round the 52 fraction bits to 7
  const uint64_t keep = frac >> 45, rem = frac & ((1ull << 45) - 1), half = 1ull << 44;
  const bool up = rem > half || (rem == half && (keep & 1));
  // exponent and mantissa fields of hi as one integer: a carry out of the mantissa
  // increments the exponent, as in the IEEE layout
  const uint32_t hfield = ((uint32_t)(E + 127) << 7) + (uint32_t)keep + (up ? 1u : 0u);
  if ((hfield >> 7) >= 255) return false;  // rounds to infinity
  hi = (uint16_t)((sign << 15) | hfield);
  // remainder x - hi in units of 2^(E - 52): rem - (up ? 2^45 : 0)
  const int64_t d = (int64_t)rem - (up ? (int64_t)(1ull << 45) : 0);
  if (d == 0) {
    lo = 0;  // x - hi = +0 under round to nearest
    return true;
  }
  const uint32_t lsign = sign ^ (d < 0 ? 1u : 0u);
  uint64_t a = (uint64_t)(d < 0 ? -d : d);
  const int msb = 63 - clz64(a);      // a in [2^msb, 2^(msb+1))
  int Elo = E - 52 + msb;             // unbiased exponent of |x - hi|
  uint64_t q;                         // 8 significant bits, 128 <= q <= 256
  if (msb > 7) {
    const int sh = msb - 7;
    q = a >> sh;
    const uint64_t r = a & ((1ull << sh) - 1), h = 1ull << (sh - 1);
    if (r > h || (r == h && (q & 1))) ++q;
  } else {
    q = a << (7 - msb);
  }
  if (q == 256) {
    q = 128;
    ++Elo;
  }
  if (Elo < -126) return false;  // lo would be subnormal
  lo = (uint16_t)((lsign << 15) | ((uint32_t)(Elo + 127) << 7) | (uint32_t)(q & 0x7F));
  return true;
}

// Bits of the binary32 value nearest to |x| (ties to even), from the bits of x; false
// outside the binary32 normal range (callers convert those).
FORTE_HD bool f32_abs_bits(double x, uint32_t &bits) {
  const uint64_t b = f64_bits(x);
  const int e = (int)((b >> 52) & 0x7FF);
  const uint64_t frac = b & ((1ull << 52) - 1);
  if (e == 0 && frac == 0) {
    bits = 0;
    return true;
  }
  const int E = e - 1023;
  if (e == 0 || E < -126 || E > 127) return false;
  const uint64_t keep = frac >> 29, rem = frac & ((1ull << 29) - 1), half = 1ull << 28;
  const bool up = rem > half || (rem == half && (keep & 1));
  bits = ((uint32_t)(E + 127) << 23) + (uint32_t)keep + (up ? 1u : 0u);
  return (bits >> 23) < 255;
}

}  // namespace forte
