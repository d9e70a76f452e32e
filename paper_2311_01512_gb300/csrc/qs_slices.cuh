// Integer slicing of FP64 operands for exact products on the bf16 tensor cores
// (the Ozaki scheme: Ozaki, Ogita, Oishi and Rump, "Error-free transformations
// of matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59 (2012)).
//
// A double x in a row (or column) whose largest biased exponent is emax becomes
// the integer V = x 2^(48 - Emax) rounded (|V| <= 2^49, Emax = emax - 1023),
// written as seven balanced digits
//   V = sum_{s=0..6} d_s 2^(42 - 7 s),   |d_0| <= 128,  -64 <= d_s <= 63 (s >= 1).
// The digits come from one 64-bit addition: with C = 64 sum_{s=1..6} 2^(42-7s),
// the unsigned 7-bit fields of W = V + C at bits 42 - 7s are d_s + 64 and the
// arithmetic top part W >> 42 is d_0.  Every digit is exact in bf16.  (The
// code keeps 2W + (0 or 1), whose fields are one bit higher, to save the
// final halving of the rounding step.)
//
// Slice products: for K <= 64 terms, sum_k a_s b_t is an integer below 2^20 in
// magnitude, and a level L = s + t (at most 7 pairs) stays below 2^22
// (2 * 64 * 128 * 64 + 5 * 64 * 64 * 64 at L = 6), so FP32 accumulation is
// exact and adding 1.5 * 2^23 puts the level's integer in the low significand
// bits.  The levels L = 0..6 are recombined modulo 2^64 from those bit
// patterns; the true value fits in 63 bits, so the wrap-around is exact.
//
// Host and device code (the host build is checked on the CPU).
#pragma once

#include <cstdint>

#include "qs_df.cuh"

namespace qsoz {

constexpr int kSlices = 7;

// C = 64 sum_{s=1..6} 2^(42-7s)
constexpr uint64_t kBal =
    64ull * ((1ull << 35) + (1ull << 28) + (1ull << 21) + (1ull << 14) + (1ull << 7) + 1ull);

// 0x4B400000 = bits of 1.5 * 2^23; the level offsets summed over the weights
// 2^(7(6-L)), modulo 2^64.
constexpr uint64_t kLevelOffset =
    0x4B400000ull * ((1ull << 42) + (1ull << 35) + (1ull << 28) + (1ull << 21) + (1ull << 14) + (1ull << 7) + 1ull);

QS_HD int biased_exp(uint32_t hw) { return (int)((hw >> 20) & 0x7FFu); }

// Lower bound of the exponent maximum (biased) of a row or column: entries
// below 2^(54 - 1023) = 2^-969 are sliced on that grid, and zeros and
// subnormals (whose implicit bit is wrongly set below) always shift out
// entirely, since their shift is then at least 57.
constexpr int kEmaxFloor = 54;

// Arithmetic right shift of a 64-bit value; amounts above 63 give the sign
// fill (PTX shr clamps the amount), which the host version matches.
QS_HD int64_t shr_s64(int64_t x, int sh) {
#if defined(__CUDA_ARCH__)
  int64_t r;
  asm("shr.s64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(sh));
  return r;
#else
  return x >> (sh > 63 ? 63 : sh);
#endif
}

// T = floor(2 x 2^(48 - Emax)) + 2C + 1 for the double with words (hw, lw),
// with emax >= max(its biased exponent, kEmaxFloor).  T is 2W or 2W + 1 for
// W = V + C, V = x 2^(48 - Emax) rounded half up (toward +infinity, so the
// rounding error does not depend on the sign of x); the digit fields of W
// sit one bit higher in T.  Zeros and subnormals give V = 0.
QS_HD uint64_t fixed_t(uint32_t hw, uint32_t lw, int emax) {
  const int sh = emax - biased_exp(hw) + 3;      // leaves one bit below the units
  const uint64_t m = (((uint64_t)(hw & 0xFFFFFu) | 0x100000u) << 32) | lw;
  const uint64_t smask = (uint64_t)(int64_t)((int32_t)hw >> 31);
  const int64_t ms = (int64_t)((m ^ smask) - smask);      // signed significand
  return (uint64_t)(shr_s64(ms, sh) + (int64_t)(2 * kBal + 1));
}

// Balanced digit s of W = T >> 1 (integer form, for checks).
QS_HD int digit_t(uint64_t t, int s) {
  if (s == 0) return (int)((int64_t)t >> 43);
  return (int)((t >> (43 - 7 * s)) & 127u) - 64;
}

// The seven digits as floats (exact small integers).
QS_HD void digit_floats_t(uint64_t t, float* f) {
  const uint32_t lo = (uint32_t)t, hi = (uint32_t)(t >> 32);
  const uint32_t d0 = (uint32_t)((int32_t)hi >> 11);
  f[0] = qsdf::u2f(0x4B400000u + d0) - 12582912.0f;
  f[1] = qsdf::u2f(0x4B400000u | ((hi >> 4) & 127u)) - 12582976.0f;
  f[2] = qsdf::u2f(0x4B400000u | ((uint32_t)(t >> 29) & 127u)) - 12582976.0f;
  f[3] = qsdf::u2f(0x4B400000u | ((lo >> 22) & 127u)) - 12582976.0f;
  f[4] = qsdf::u2f(0x4B400000u | ((lo >> 15) & 127u)) - 12582976.0f;
  f[5] = qsdf::u2f(0x4B400000u | ((lo >> 8) & 127u)) - 12582976.0f;
  f[6] = qsdf::u2f(0x4B400000u | ((lo >> 1) & 127u)) - 12582976.0f;
}

// sum_L level_L 2^(7(6-L)) from the bit patterns b_L of (level_L + 1.5 * 2^23).
QS_HD int64_t combine_levels(const uint32_t* b) {
  uint64_t acc = (uint64_t)b[6] - kLevelOffset;
  acc += (uint64_t)b[5] * 128u;
  acc += (uint64_t)b[4] * 16384u;
  acc += (uint64_t)b[3] * 2097152u;
  acc += (uint64_t)b[2] * 268435456u;
  acc += (uint64_t)(b[1] * 8u + b[0] * 1024u) << 32;
  return (int64_t)acc;
}

// ---------------------------------------------------------------------------
// Eight slices (56 bits, at least the 53 of IEEE double).  A double x in a row
// or column of largest biased exponent emax becomes V = x 2^(55 - Emax)
// rounded (|V| <= 2^56), with eight balanced digits
//   V = sum_{s=0..7} d_s 2^(49 - 7 s),   |d_0| <= 128,  -64 <= d_s <= 63,
// taken from W = V + C8, C8 = 64 sum_{s=1..7} 2^(49-7s), as above.  Levels
// L = s + t <= 7 stay exact in FP32 for K <= 64 (level 7: two products with
// d_0, 2 64 128 64, and six others, 6 64 64 64: below 2.5 2^20).  The full
// sum of levels, sum_L level_L 2^(7(7-L)), reaches 2^71, so the recombination
// keeps it divided by 2^8: levels 0..5 with the integer weights 2^(41-7L)
// modulo 2^64 (the true value is below 2^61), plus
// floor((128 level_6 + level_7) / 2^8).
// ---------------------------------------------------------------------------
constexpr int kSlices8 = 8;
constexpr uint64_t kBal8 =
    64ull * ((1ull << 42) + (1ull << 35) + (1ull << 28) + (1ull << 21) + (1ull << 14) + (1ull << 7) + 1ull);
constexpr uint64_t kLevelOffset8 =
    0x4B400000ull * ((1ull << 41) + (1ull << 34) + (1ull << 27) + (1ull << 20) + (1ull << 13) + (1ull << 6));

// T = floor(2 x 2^(55 - Emax)) + 2 C8 + 1 (fields of W one bit higher).
QS_HD uint64_t fixed_t8(uint32_t hw, uint32_t lw, int emax) {
  const int sh = emax - biased_exp(hw);          // >= 0; the significand is pre-shifted by 4
  const uint64_t m = (((uint64_t)(hw & 0xFFFFFu) | 0x100000u) << 32) | lw;
  const uint64_t smask = (uint64_t)(int64_t)((int32_t)hw >> 31);
  const int64_t ms = (int64_t)((m ^ smask) - smask);
  return (uint64_t)(shr_s64((int64_t)((uint64_t)ms << 4), sh) + (int64_t)(2 * kBal8 + 1));
}

QS_HD int digit_t8(uint64_t t, int s) {
  if (s == 0) return (int)((int64_t)t >> 50);
  return (int)((t >> (50 - 7 * s)) & 127u) - 64;
}

QS_HD void digit_floats_t8(uint64_t t, float* f) {
  const uint32_t lo = (uint32_t)t, hi = (uint32_t)(t >> 32);
  const uint32_t d0 = (uint32_t)((int32_t)hi >> 18);
  f[0] = qsdf::u2f(0x4B400000u + d0) - 12582912.0f;
  f[1] = qsdf::u2f(0x4B400000u | ((hi >> 11) & 127u)) - 12582976.0f;
  f[2] = qsdf::u2f(0x4B400000u | ((hi >> 4) & 127u)) - 12582976.0f;
  f[3] = qsdf::u2f(0x4B400000u | ((uint32_t)(t >> 29) & 127u)) - 12582976.0f;
  f[4] = qsdf::u2f(0x4B400000u | ((lo >> 22) & 127u)) - 12582976.0f;
  f[5] = qsdf::u2f(0x4B400000u | ((lo >> 15) & 127u)) - 12582976.0f;
  f[6] = qsdf::u2f(0x4B400000u | ((lo >> 8) & 127u)) - 12582976.0f;
  f[7] = qsdf::u2f(0x4B400000u | ((lo >> 1) & 127u)) - 12582976.0f;
}

// floor(sum_L level_L 2^(7(7-L)) / 2^8) from the bit patterns b_L of (level_L + 1.5 * 2^23).
QS_HD int64_t combine_levels8(const uint32_t* b) {
  uint64_t acc = (uint64_t)b[5] * 64u - kLevelOffset8;
  acc += (uint64_t)b[4] * 8192u;
  acc += (uint64_t)b[3] * 1048576u;
  acc += (uint64_t)b[2] * 134217728u;
  acc += ((uint64_t)b[1] << 34) + ((uint64_t)b[0] << 41);
  const int32_t low = ((int32_t)(b[6] - 0x4B400000u) * 128 + (int32_t)(b[7] - 0x4B400000u)) >> 8;
  return (int64_t)(acc + (uint64_t)(int64_t)low);
}

}  // namespace qsoz
