// Exact digit-slice products on the BF16 tensor cores (the splitting scheme of
// Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59 (2012) 95, with integer
// slices): definitions shared by the tensor-core 2-RDM Gram and the FP64-class
// alpha-beta sigma.
//
// A fixed-point integer |X| <= 2^45 is written as six balanced base-256 digits
// X = sum_i d_i 256^(6-i), |d_1| <= 32, d_2..d_6 in [-128, 127]; each digit is
// exact in BF16.  Over K <= 64 products the level sums
//   L_t = sum_{i+j=t} sum_k a_i(k) b_j(k),   t = 2..8,
// stay below 2^23 and are summed exactly by the FP32 tensor-core accumulator.
// Levels t > 8 are dropped (weight at most 2^-49.99 of K times the product of
// the two operand bounds, for worst-case digits).  The epilogue folds the levels into one 64-bit integer in
// units of 2^6 L_8 (L_8 carries weight 256^4 = 2^32 in the product X_a X_b).
#pragma once

#include <stdint.h>

#include "tc_ptx.cuh"

namespace forte {

constexpr int OZ_DIGITS = 6;
constexpr int OZ_TMAX = 8;
constexpr int OZ_XBITS = 45;  // |X| <= 2^45 after scaling

// Level shifts into the 64-bit accumulator (units of 2^6 L_8): L_t carries
// weight 2^(8(8-t)) L_8, so the shift is 8(8-t) - 6; L_7 arrives in units of 2.
__host__ __device__ constexpr int oz_shift(int t) { return t == 7 ? 3 : 8 * (8 - t) - 6; }
// Sum over levels 2..7 of (magic bits << shift), modulo 2^64: the magic-number
// rounding adds 0x4B400000 (1.5 2^23) or 0x4BC00000 (1.5 2^24) to every level.
__host__ __device__ constexpr unsigned long long oz_bias() {
  unsigned long long b = 0;
  for (int t = 2; t <= 6; ++t) b += (unsigned long long)0x4B400000u << oz_shift(t);
  b += (unsigned long long)0x4BC00000u << oz_shift(7);
  return b;
}

// FP32 bits of (byte k of w) - 128: the byte is placed under the exponent of
// 1.5 2^23 and the bias is subtracted exactly.
__device__ __forceinline__ uint32_t oz_dig(uint32_t w, uint32_t k) {
  return __float_as_uint(__uint_as_float(__byte_perm(w, 0x4B400000u, 0x7650u | k)) - 12583040.0f);
}

// Fold level T of one product (the FP32 accumulator bits) into acc: the level is
// rounded to an integer by the magic-number addition and shifted into place
// (modulo 2^64; the caller subtracts oz_bias() once per folded chunk).
template <int T>
__device__ __forceinline__ void oz_acc_level(unsigned long long &acc, uint32_t fbits) {
  const float f = __uint_as_float(fbits);
  if constexpr (T <= 6) {
    const uint32_t m = __float_as_uint(f + 12582912.0f);
    if constexpr (oz_shift(T) >= 32)
      acc += (unsigned long long)(m << (oz_shift(T) - 32)) << 32;  // high word only
    else
      acc += (unsigned long long)m * (1ull << oz_shift(T));  // one wide multiply-add
  } else if constexpr (T == 7) {
    acc += (unsigned long long)__float_as_uint(f + 25165824.0f) * (1ull << oz_shift(7));
  } else {
    const int v = (int)(__float_as_uint(f + 25165824.0f) - 0x4BC00000u);  // L_8 / 2
    acc += (unsigned long long)(long long)((v + 16) >> 5);
  }
}

// The MMA chain of level LV: for every digit pair (i, j), i + j = LV, and every
// 16-deep K step, D (+)= A_i B_j^T.  a0 / b0 are the shared-memory descriptors of
// digit slice 1 at K offset 0; slices lie ASL / BSL descriptor units (16 bytes)
// apart and a K step is 2 units (32 bytes) inside the 128-byte swizzled rows.
// Fully unrolled, so that each MMA costs the issuing thread one descriptor
// addition per operand.
template <int LV, int ASL, int BSL, int NKS>
__device__ __forceinline__ void oz_issue_level(uint32_t d, uint64_t a0, uint64_t b0, uint32_t idesc) {
  constexpr int lo = LV - OZ_DIGITS > 1 ? LV - OZ_DIGITS : 1;
  constexpr int hi = LV - 1 < OZ_DIGITS ? LV - 1 : OZ_DIGITS;
#pragma unroll
  for (int ks = 0; ks < NKS; ++ks)
#pragma unroll
    for (int ia = lo; ia <= hi; ++ia)
      mma_issue<FORTE_BF16X2>(d, a0 + (uint64_t)((ia - 1) * ASL + 2 * ks), b0 + (uint64_t)((LV - ia - 1) * BSL + 2 * ks),
                              idesc, (ks == 0 && ia == lo) ? 0u : 1u);
}

}  // namespace forte
