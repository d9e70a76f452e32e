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


// ---------------------------------------------------------------------------
// Offset-packed amplitude digits.  For s >= 1 the unsigned field d_s + 64 of
// T sits in 7 bits; the bf16 number whose exponent is 2^7 and whose stored
// significand is that field equals 128 + (d_s + 64) = d_s + 192, with bit
// pattern 0x4300 | field.  So the (re, im) word of digit s is two shifted
// fields and one constant, with no float arithmetic.  The offset adds
// 192 sum_k b_t(k, n) to each level L = s + t with s >= 1; the tensor-core
// kernel starts each accumulator (with one initialising MMA) at
//   P_L(n) = M - 192 sum_{t=0..L-1} sum_k b_t(k, n),
// M = 0 (K = 64), or M = 1.25 2^23 (K <= 32), where the accumulator then ends
// as the FP32 number magic + level whose bit pattern is 0x4B200000 + level.
// Every partial sum stays an integer below 2^24 in magnitude (checked on the
// host over the extreme digits), so the accumulation stays exact.  The top
// digit d_0 is signed and keeps the float path.
// ---------------------------------------------------------------------------
constexpr int kDigitOffset = 192;
constexpr float kPreMagic = 10485760.0f;        // 1.25 2^23
constexpr uint32_t kPreMagicBits = 0x4B200000u;
constexpr uint32_t kFaddMagicBits = 0x4B400000u;  // 1.5 2^23, added in the epilogue when M = 0

// bit position in T of digit s >= 1 (seven or eight slices)
template <int KS>
QS_HD constexpr int digit_pos(int s) { return 1 + 7 * (KS - 1 - s); }

// packed bf16 pair (re in bits 0..15, im in 16..31) of digit S >= 1
template <int KS, int S>
QS_HD uint32_t packed_pair(uint64_t tre, uint64_t tim) {
  constexpr int p = digit_pos<KS>(S);
  uint32_t im;
  if constexpr (p >= 16)
    im = (uint32_t)(tim >> (p - 16)) & 0x7F0000u;
  else
    im = (uint32_t)(tim << (16 - p)) & 0x7F0000u;
  return 0x43004300u | ((uint32_t)(tre >> p) & 127u) | im;
}

// P = p[0] + 256 p[1] + 65536 p[2] with |p[i]| <= 256 (exact in bf16), each
// part rounded to nearest, for |P| < 2^24: the B column of the initialising
// MMA, whose A rows are (1, 256, 65536).
QS_HD void split_start(int P, int* p) {
  p[2] = (P + (P >= 0 ? 32768 : -32768)) / 65536;
  const int r = P - 65536 * p[2];
  p[1] = (r + (r >= 0 ? 128 : -128)) / 256;
  p[0] = r - 256 * p[1];
}

// byte permute (PTX prmt / __byte_perm): byte i of the result is byte
// ((sel >> 4i) & 7) of the eight bytes (y:x)
QS_HD uint32_t byte_perm(uint32_t x, uint32_t y, uint32_t sel) {
#if defined(__CUDA_ARCH__)
  return __byte_perm(x, y, sel);
#else
  const uint64_t v = ((uint64_t)y << 32) | x;
  uint32_t r = 0;
  for (int i = 0; i < 4; ++i) r |= (uint32_t)((v >> (8 * ((sel >> (4 * i)) & 7))) & 0xFF) << (8 * i);
  return r;
#endif
}

// packed_pair through one byte permute where the field's byte-aligned 16-bit
// window lies in one 32-bit word of T (all digits but the one at bit 29): the
// re and im windows side by side, one shift, one mask-and-or.
template <int KS, int S>
QS_HD uint32_t packed_pair_fast(uint64_t tre, uint64_t tim) {
  constexpr int p = digit_pos<KS>(S);
  constexpr int wb = p / 8;                 // first byte of the window in T
  constexpr int r = p - 8 * wb;             // the field's offset in it
  if constexpr (wb == 3) {
    return packed_pair<KS, S>(tre, tim);
  } else {
    constexpr int hiw = wb >= 4;             // which 32-bit word
    constexpr uint32_t B = (uint32_t)(wb - 4 * hiw);
    constexpr uint32_t sel = B | ((B + 1) << 4) | ((B + 4) << 8) | ((B + 5) << 12);
    const uint32_t xr = (uint32_t)(hiw ? tre >> 32 : tre), xi = (uint32_t)(hiw ? tim >> 32 : tim);
    const uint32_t x = byte_perm(xr, xi, sel);
    return ((r ? x >> r : x) & 0x007F007Fu) | 0x43004300u;
  }
}

// packed words of digits S..KS-1 into w[S..KS-1] (byte-permute form)
template <int KS, int S = 1>
QS_HD void packed_digits_fast(uint64_t tre, uint64_t tim, uint32_t* w) {
  w[S] = packed_pair_fast<KS, S>(tre, tim);
  if constexpr (S + 1 < KS) packed_digits_fast<KS, S + 1>(tre, tim, w);
}

// packed words of digits S..KS-1 into w[S..KS-1]
template <int KS, int S = 1>
QS_HD void packed_digits(uint64_t tre, uint64_t tim, uint32_t* w) {
  w[S] = packed_pair<KS, S>(tre, tim);
  if constexpr (S + 1 < KS) packed_digits<KS, S + 1>(tre, tim, w);
}

// T of a double for seven or eight slices
template <int KS>
QS_HD uint64_t fixed_ks(uint32_t hw, uint32_t lw, int emax) {
  if constexpr (KS == 8)
    return fixed_t8(hw, lw, emax);
  else
    return fixed_t(hw, lw, emax);
}

// top digit d_0 of T as an exact float
template <int KS>
QS_HD float top_digit(uint64_t t) {
  const uint32_t d0 = (uint32_t)((int32_t)(uint32_t)(t >> 32) >> (KS == 8 ? 18 : 11));
  return qsdf::u2f(0x4B400000u + d0) - 12582912.0f;
}

// sum_L level_L 2^(7(KS-1-L)) (divided by 2^8, rounded down, for eight
// slices) from the bit patterns b_L = mb + level_L, merging adjacent levels
// in 32 bits first: q = 128 level_L + level_(L+1) stays below 2^28 in magnitude.
template <int KS>
QS_HD int64_t combine_pairs(const uint32_t* b, uint32_t mb) {
  const uint32_t off = 129u * mb;
  const int32_t q0 = (int32_t)(b[0] * 128u + b[1] - off);
  const int32_t q1 = (int32_t)(b[2] * 128u + b[3] - off);
  const int32_t q2 = (int32_t)(b[4] * 128u + b[5] - off);
  if constexpr (KS == 8) {
    const int32_t q3 = (int32_t)(b[6] * 128u + b[7] - off);
    return (int64_t)((uint64_t)(int64_t)q0 << 34) + (int64_t)((uint64_t)(int64_t)q1 << 20) +
           (int64_t)q2 * 64 + (int64_t)(q3 >> 8);
  } else {
    const int32_t l6 = (int32_t)(b[6] - mb);
    return (int64_t)((uint64_t)(int64_t)q0 << 35) + (int64_t)((uint64_t)(int64_t)q1 << 21) +
           (int64_t)q2 * 128 + (int64_t)l6;
  }
}

// The same with the merged words used unsigned: r = 128 b_L + b_(L+1) equals
// q + 129 MB mod 2^32, and for the level bounds of the kernels it does not
// wrap (MB = kPreMagicBits, K <= 32, |level| <= 1310720: r within
// 0xDB200000 +- 1.7e8; MB = kFaddMagicBits, K <= 64, |level| <= 2621440: r
// within 0xEB400000 +- 3.39e8 < 2^32), so the offsets leave as one 64-bit
// constant (divisible by 2^8 where the floor applies).
template <int KS, uint32_t MB>
QS_HD int64_t combine_pairs_u(const uint32_t* b) {
  constexpr uint64_t off = (129ull * MB) & 0xFFFFFFFFull;
  const uint32_t r0 = b[0] * 128u + b[1], r1 = b[2] * 128u + b[3], r2 = b[4] * 128u + b[5];
  if constexpr (KS == 8) {
    static_assert((off & 255u) == 0, "floor of the last word");
    constexpr uint64_t C = off * ((1ull << 34) + (1ull << 20) + (1ull << 6)) + (off >> 8);
    const uint32_t r3 = b[6] * 128u + b[7];
    return (int64_t)(((uint64_t)r0 << 34) + ((uint64_t)r1 << 20) + ((uint64_t)r2 << 6) + (uint64_t)(r3 >> 8) - C);
  } else {
    constexpr uint64_t C = off * ((1ull << 35) + (1ull << 21) + (1ull << 7)) + MB;
    return (int64_t)(((uint64_t)r0 << 35) + ((uint64_t)r1 << 21) + ((uint64_t)r2 << 7) + (uint64_t)b[6] - C);
  }
}

}  // namespace qsoz
