// Double-float ("df") arithmetic for complex128 amplitudes on the FP32 pipes.
//
// GB300 runs FP64 FMA at ~1.2 TFLOP/s but FP32 FMA at ~70 TFLOP/s, and its
// f64<->f32 conversion instructions run at the FP64 rate.  So a complex128
// value x is split into two floats by integer bit operations only:
//   hi = x with its significand truncated to 24 bits,
//   lo = the rest of the significand rounded to 23 bits,
// so |x - (hi + lo)| <= 2^-47 |x|.  Both the split and the join round to
// nearest with ties to even, so the conversions carry no systematic bias.  The arithmetic is done on (hi, lo) pairs with
// error-free FP32 transformations (Dekker/Knuth TwoProd via FMA, TwoSum,
// Fast2Sum), and the result is joined back into an IEEE double by integer
// operations.  Relative error of one dot product: a few units of 2^-46.
//
// Range: the relative error bound holds for 2^-80 <= |x| < 2^128.  Below 2^-80
// the low part is an FP32 subnormal and is dropped, and below 2^-103 x is
// flushed to zero: the absolute error stays under 2^-103 there.
//
// The same code compiles for the host (integer logic tested on the CPU) and
// the device.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define QS_HD __host__ __device__ __forceinline__
#else
#define QS_HD inline
#endif

namespace qsdf {

struct df {
  float h, l;
};

QS_HD uint32_t f2u(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(f);
#else
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
#endif
}

QS_HD float u2f(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, 4);
  return f;
#endif
}

QS_HD void d2w(double x, uint32_t& hw, uint32_t& lw) {
#if defined(__CUDA_ARCH__)
  hw = (uint32_t)__double2hiint(x);
  lw = (uint32_t)__double2loint(x);
#else
  uint64_t u;
  std::memcpy(&u, &x, 8);
  hw = (uint32_t)(u >> 32);
  lw = (uint32_t)u;
#endif
}

QS_HD double w2d(uint32_t hw, uint32_t lw) {
#if defined(__CUDA_ARCH__)
  return __hiloint2double((int)hw, (int)lw);
#else
  const uint64_t u = ((uint64_t)hw << 32) | lw;
  double x;
  std::memcpy(&x, &u, 8);
  return x;
#endif
}

// (hi:lo) << 3, top word
QS_HD uint32_t funnel3(uint32_t lo, uint32_t hi) {
#if defined(__CUDA_ARCH__)
  return __funnelshift_l(lo, hi, 3);
#else
  return (hi << 3) | (lo >> 29);
#endif
}

QS_HD float fmaf_(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return __builtin_fmaf(a, b, c);
#endif
}

// Split an IEEE double into (hi, lo) floats, integer operations only.
// hi: sign, exponent e - 896 (re-biased), top 23 stored significand bits.
// lo: the remaining 29 significand bits rounded to 23, as the difference of
// two floats that share hi's sign and the exponent 23 below hi's (exact; a
// rounding carry into the exponent field still gives the right value).
QS_HD df split(double x) {
  uint32_t hw, lw;
  d2w(x, hw, lw);
  // bits 31..23 of the funnel shift hold e mod 512; adding 128 there gives
  // e - 896 for 896 <= e < 1152, with bit 31 clear.
  const uint32_t t = funnel3(lw, hw) + 0x40000000u;
  const uint32_t hb = t | (hw & 0x80000000u);
  const uint32_t base = (hb & 0xFF800000u) - 0x0B800000u;  // exponent - 23
  // 29 low significand bits rounded to 23, ties to even (no bias): <= 2^23
  const uint32_t r29 = lw & 0x1FFFFFFFu;
  const uint32_t mant = (r29 + 31u + ((r29 >> 6) & 1u)) >> 6;
  df r;
  r.h = u2f(hb);
  r.l = u2f(base + mant) - u2f(base);
  // e < 920 (|x| < 2^-103, zeros and subnormals included): flush to zero
  if ((hw << 1) < (920u << 21)) {
    r.h = 0.0f;
    r.l = 0.0f;
  }
  return r;
}

// Join a normalised pair (|l| <= ulp(h)/2, as left by dot_result) into an
// IEEE double: h + l rounded to nearest, ties to even, integer operations only.
// h has 24 significant bits, so the last bit of the result is the last bit of
// l in units of the double's last place; rounding that to even rounds the sum.
QS_HD double join(df v) {
  const uint32_t hb = f2u(v.h), lb = f2u(v.l);
  const int eh = (int)((hb >> 23) & 0xFFu);
  const int el = (int)((lb >> 23) & 0xFFu);
  // h as a double: sign | (eh + 896) << 20 | significand >> 3 : significand << 29
  uint32_t dh = (((hb & 0x7FFFFFFFu) >> 3) + (896u << 20)) | (hb & 0x80000000u);
  uint32_t dl = hb << 29;
  // l in units of the double's last place 2^(Eh - 52): significand shifted by el - eh + 29
  const uint32_t ml = (lb & 0x7FFFFFu) | 0x800000u;
  const int sh = el - eh + 29;
  // normalised pairs have sh <= 5, so li < 2^29 never reaches h's significand
  uint32_t li;
  if (sh >= 0) {
    li = ml << sh;
  } else if (sh < -24) {
    li = 0u;
  } else {
    const int k = -sh;
    li = (ml + (1u << (k - 1)) - 1u + ((ml >> k) & 1u)) >> k;
  }
  if (el == 0) li = 0;                     // l is zero (or subnormal)
  const bool opposite = ((hb ^ lb) >> 31) != 0;
  // below a power of two the last place halves
  if (opposite && (hb & 0x7FFFFFu) == 0) li <<= 1;
  uint64_t mag = ((uint64_t)(dh & 0x7FFFFFFFu) << 32) | dl;
  mag = opposite ? mag - li : mag + li;
  dh = (uint32_t)(mag >> 32) | (dh & 0x80000000u);
  dl = (uint32_t)mag;
  if (eh == 0) {                           // h is zero (or subnormal): so is the sum
    dh = hb & 0x80000000u;
    dl = 0;
  }
  return w2d(dh, dl);
}

// Exact float -> double by bit construction (no FP64 conversion instruction).
// The arithmetic shift keeps the sign in bit 31 and clears bits 28..30, so
// the high word is sign | (exponent - 127 + 1023) << 20 | significand >> 3
// once the exponent bias 896 << 20 is added; zeros (exponent field 0) get no
// bias and stay signed zeros.  FP32 subnormals (|f| < 2^-126) come out as
// double subnormals below 2^-1022 instead of their value: an absolute error
// under 2^-126.
QS_HD double to_double(float f) {
  const uint32_t b = f2u(f);
  const uint32_t bias = (b & 0x7F800000u) ? (896u << 20) : 0u;
  const uint32_t dh = ((uint32_t)((int32_t)b >> 3) & 0x8FFFFFFFu) + bias;
  return w2d(dh, b << 29);
}

// Constants (gate-matrix entries) are split exactly on the host: h = (float)x,
// l = (float)(x - h); |x - (h + l)| <= 2^-48 |x|.
inline df split_const(double x) {
  df r;
  r.h = (float)x;
  r.l = (float)(x - (double)r.h);
  return r;
}

// Accumulator of sum_k c_k v_k: the exact running sum of the hi*hi products
// (s plus the TwoSum errors gathered in lo), the FMA errors of those
// products, and the cross terms c.h*v.l + c.l*v.h.  c.l*v.l (2^-48 relative)
// is dropped.
struct dot_acc {
  float s, lo;
};

QS_HD dot_acc dot_first(df c, df v) {
  dot_acc a;
  const float p = c.h * v.h;
  a.lo = fmaf_(c.h, v.h, -p);
  a.lo = fmaf_(c.h, v.l, a.lo);
  a.lo = fmaf_(c.l, v.h, a.lo);
  a.s = p;
  return a;
}

QS_HD void dot_add(dot_acc& a, df c, df v) {
  const float p = c.h * v.h;
  float lo = fmaf_(c.h, v.h, -p);
  lo = fmaf_(c.h, v.l, lo);
  lo = fmaf_(c.l, v.h, lo);
  // TwoSum(s, p)
  const float s2 = a.s + p;
  const float bb = s2 - a.s;
  const float err = (a.s - (s2 - bb)) + (p - bb);
  a.s = s2;
  a.lo += lo + err;
}

// TwoSum of the accumulator into a normalised pair (|l| <= ulp(h)/2 even when
// the hi sum cancels and lo dominates).
QS_HD df dot_result(const dot_acc& a) {
  df r;
  r.h = a.s + a.lo;
  const float bb = r.h - a.s;
  r.l = (a.s - (r.h - bb)) + (a.lo - bb);
  return r;
}

// The accumulated value s + lo as an IEEE double, rounded once (one FP64 add
// of two exactly converted floats).  The kernels end every dot product here:
// a single DADD is cheaper on GB300 than an integer join, and the FP64 pipe is
// otherwise idle in these kernels.
QS_HD double finish(const dot_acc& a) { return to_double(a.s) + to_double(a.lo); }

// Product of a df value with a plain float constant whose value is exact in
// 24 bits (used for +-1 and 0 multipliers; cheap).
QS_HD df neg(df v) {
  df r;
  r.h = -v.h;
  r.l = -v.l;
  return r;
}

}  // namespace qsdf
