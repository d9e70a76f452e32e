// Block fixed-point ("fx") arithmetic for complex128 amplitudes: exact
// integer products on the 32-bit integer multipliers, one rounding per output.
//
// Why: GB300 runs FP64 FMA at about 1/70 of its FP32 rate, so a plain FP64
// one-target gate is FP64-pipe bound (about three times the HBM time at 30
// qubits).  Double-float (qs_df.cuh) keeps the HBM rate but only 47 bits.
// This form keeps at least the 53 bits of IEEE double and still moves
// memory at the HBM rate.
//
// Representation.  The doubles x_k that one output combines (the real and
// imaginary parts of the amplitudes of a pair, a group or a single amplitude)
// share the exponent ex = the largest biased exponent among them and become
// signed integers
//     X_k = trunc(x_k 2^(1082 - ex)),   |X_k| < 2^60,
// exact for every x_k within 7 binades of the largest (the largest itself
// has 53 significant bits and 7 zero bits below them), truncated toward zero
// by less than one unit 2^(ex - 1082) otherwise.  Subnormals (below
// 2^-1022) carry an error of at most their own size.  The constants of a row
// group (gate-matrix entries, cos/sin of a gadget, channel coefficients) share
// their largest biased exponent em in the same way, rounded to nearest on the
// host:
//     M = round(m 2^(1082 - em)),   |M| < 2^60.
// Every integer is split into two 30-bit parts, X = h 2^30 + l: a constant as
// h = floor(M / 2^30) in [-2^30, 2^30), l = M mod 2^30 in [0, 2^30); an
// amplitude's integer as its magnitude's parts, both carrying its sign
// (|h|, |l| < 2^30).  Every product of parts is below 2^60 in magnitude.
//
// Products.  x m = X M 2^(ex + em - 2164) and
//     X M = h_x h_m 2^60 + (h_x l_m + l_x h_m) 2^30 + l_x l_m.
// An output sum_k x_k m_k over K <= 4 terms accumulates A = sum h_x h_m and
// B = sum (h_x l_m + l_x h_m) exactly in 64-bit integers (|A| < 2^62,
// |B| < 2^63), each product as one mad.lo.cc / madc.hi pair of 32-bit
// multiplies with carry (about three times the rate of a 32x32->64
// multiply-add on this GPU).  The sum l_x l_m (< 4 2^60, below one unit of A
// in total) is dropped, and
//     V = A + floor(B / 2^30),     y = V 2^(ex + em - 2104)
// is rounded once to double (int64 -> double, round to nearest even) and
// scaled by adding to the exponent field.
//
// Error of one output y = sum_k x_k m_k (K <= 4), with X = max_k |x_k| and
// Mx = max_k |m_k| (so 2^(ex-1023) <= X and 2^(em-1023) <= Mx):
//     |fx(y) - y| <= 2^-53 |y| + 2^-55 X Mx    (plus flushes below 2^-1022)
// from: truncation of the x_k (< 2^(ex-1082) each, times |m_k|), rounding of
// the m_k (<= 2^(em-1083) each, times |x_k|), the dropped l_x l_m and floor
// (< 5 units of 2^(ex+em-2104) = 5 2^-58 2^(ex+em-2046)), then the final
// rounding.
//
// An output over K <= 8 terms (the eight real parts of the four amplitudes of
// a two-target gate) accumulates its terms 0..3 and 4..7 in two such
// accumulators, so every partial sum keeps the bounds above, and
//     V = A_lo + floor(B_lo / 2^30) + A_hi + floor(B_hi / 2^30),   |V| < 2^63
// (|V| is below sum_k |X_k M_k| / 2^60 + 10 <= 8 (2^60 - 2^7) + 10).  The
// error terms count as before with K = 8 and two floors, (7 K + 8) 2^-60 X Mx:
//     |fx(y) - y| <= 2^-53 |y| + 2^-54 X Mx    (K <= 8).
// The host test tests/host/fx_check.cpp checks both bounds against exact
// rational arithmetic.
//
// The same code compiles for the host (tested on the CPU) and the device.
#pragma once

#include <cstdint>

#include "qs_df.cuh"   // QS_HD, d2w, w2d

namespace qsfx {

constexpr int kShift = 1082;   // x = X 2^(ex - kShift)
constexpr int kFinish = 2104;  // y = V 2^(ex + em - kFinish)

struct Part {
  int32_t h, l;   // X = h 2^30 + l, |h|, |l| <= 2^30
};

// 64-bit accumulators A (h h) and B (cross terms).
struct Acc {
  uint32_t alo, blo;
  int32_t ahi, bhi;
};

QS_HD int expo(uint32_t hw) { return (int)((hw >> 20) & 0x7FFu); }
QS_HD int expo_of(double x) {
  uint32_t hw, lw;
  qsdf::d2w(x, hw, lw);
  return expo(hw);
}

QS_HD Part split64(int64_t X) {
  Part p;
  p.h = (int32_t)(X >> 30);
  p.l = (int32_t)((uint32_t)X & 0x3FFFFFFFu);
  return p;
}

QS_HD uint64_t shr_u64(uint64_t x, uint32_t d) {
#if defined(__CUDA_ARCH__)
  uint64_t r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(d));   // amounts above 63 give 0
  return r;
#else
  return d > 63 ? 0ull : x >> d;
#endif
}

// x (words hw:lw, exponent field ef = hw & 0x7FF00000) in the block whose
// largest exponent field is exf >= ef.  The sign is kept on both parts
// (|h|, |l| < 2^30; the product bounds are those of the floor split).  A zero
// gets no implicit bit; a subnormal is read with exponent 0 instead of 1 (half
// its value; it only matters when the whole block is below 2^-964).
QS_HD Part fixed_f(uint32_t hw, uint32_t lw, uint32_t ef, uint32_t exf) {
  const uint32_t hid = ef < 0x100000u ? ef : 0x100000u;   // implicit bit, none for zeros
  const uint64_t m = ((uint64_t)((hw & 0xFFFFFu) | hid) << 39) | ((uint64_t)lw << 7);
  const uint64_t mag = shr_u64(m, (exf - ef) >> 20);
  const int32_t sg = ((int32_t)hw >> 31) | 1;             // +1 or -1
  Part p;
  p.h = (int32_t)(uint32_t)(mag >> 30) * sg;
  p.l = (int32_t)((uint32_t)mag & 0x3FFFFFFFu) * sg;
  return p;
}

// x in the block of largest biased exponent ex >= its own.
QS_HD Part fixed(uint32_t hw, uint32_t lw, int ex) {
  return fixed_f(hw, lw, hw & 0x7FF00000u, (uint32_t)ex << 20);
}

QS_HD Part fixed_d(double x, int ex) {
  uint32_t hw, lw;
  qsdf::d2w(x, hw, lw);
  return fixed(hw, lw, ex);
}

// Constant m in a group of largest biased exponent em >= its own, rounded to
// nearest (ties away from zero); |M| <= 2^60.
QS_HD Part fixed_const(double x, int em) {
  uint32_t hw, lw;
  qsdf::d2w(x, hw, lw);
  const int e = expo(hw);
  const uint64_t m = ((uint64_t)((hw & 0xFFFFFu) | 0x100000u) << 39) | ((uint64_t)lw << 7);
  const int d = em - e;
  uint64_t mag = 0;
  if (e != 0 && d < 61) mag = d == 0 ? m : ((m >> (d - 1)) + 1) >> 1;
  const int64_t X = (int32_t)hw < 0 ? -(int64_t)mag : (int64_t)mag;
  return split64(X);
}

QS_HD Acc acc_zero() {
  Acc a;
  a.alo = a.blo = 0u;
  a.ahi = a.bhi = 0;
  return a;
}

// a += x m (the h h product into A, the two cross products into B).
QS_HD void mac(Acc& a, Part x, Part m) {
#if defined(__CUDA_ARCH__)
  asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\tmadc.hi.s32 %1, %2, %3, %1;"
      : "+r"(a.alo), "+r"(a.ahi) : "r"(x.h), "r"(m.h));
  asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\tmadc.hi.s32 %1, %2, %3, %1;"
      : "+r"(a.blo), "+r"(a.bhi) : "r"(x.h), "r"(m.l));
  asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\tmadc.hi.s32 %1, %2, %3, %1;"
      : "+r"(a.blo), "+r"(a.bhi) : "r"(x.l), "r"(m.h));
#else
  int64_t A = (int64_t)(((uint64_t)(uint32_t)a.ahi << 32) | a.alo);
  int64_t B = (int64_t)(((uint64_t)(uint32_t)a.bhi << 32) | a.blo);
  A += (int64_t)x.h * m.h;
  B += (int64_t)x.h * m.l + (int64_t)x.l * m.h;
  a.alo = (uint32_t)A;
  a.ahi = (int32_t)((uint64_t)A >> 32);
  a.blo = (uint32_t)B;
  a.bhi = (int32_t)((uint64_t)B >> 32);
#endif
}

QS_HD int64_t acc_value(const Acc& a) {
  const int64_t A = (int64_t)(((uint64_t)(uint32_t)a.ahi << 32) | a.alo);
  const int64_t B = (int64_t)(((uint64_t)(uint32_t)a.bhi << 32) | a.blo);
  return A + (B >> 30);
}

QS_HD double i64_to_double(int64_t v) {
#if defined(__CUDA_ARCH__)
  return __ll2double_rn(v);
#else
  return (double)v;
#endif
}

// Scaling of an output block: y = V 2^sc, sc = ex + em - 2104, applied as an
// exponent-field increment inc = sc 2^20 to the rounded V; results whose
// exponent field would fall to 0 or below (|y| < 2^-1022) are flushed to 0,
// which the single test |hw| > thr does (thr = max(-sc, 0) 2^20 + 2^20 - 1;
// it also keeps V = 0 at 0).
struct Scale {
  uint32_t inc, thr;
};
QS_HD Scale scale_for(int ex, int em) {
  const int sc = ex + em - kFinish;
  Scale s;
  s.inc = (uint32_t)sc * (1u << 20);
  const int under = sc < 0 ? (-sc < 2047 ? -sc : 2047) : 0;
  s.thr = ((uint32_t)under << 20) | 0xFFFFFu;
  return s;
}

// V rounded once to double and scaled by 2^sc.
QS_HD double finish_v(int64_t v, Scale s) {
  const double r = i64_to_double(v);
  uint32_t hw, lw;
  qsdf::d2w(r, hw, lw);
  const bool ok = (hw & 0x7FFFFFFFu) > s.thr;
  return qsdf::w2d(ok ? hw + s.inc : 0u, ok ? lw : 0u);
}

QS_HD double finish_s(const Acc& a, Scale s) { return finish_v(acc_value(a), s); }

// An output accumulated in two halves (terms 0..3 in lo, 4..7 in hi).
QS_HD double finish2_s(const Acc& lo, const Acc& hi, Scale s) { return finish_v(acc_value(lo) + acc_value(hi), s); }

// The accumulated sum as a double: V rounded once, times 2^(ex + em - 2104).
QS_HD double finish(const Acc& a, int ex, int em) { return finish_s(a, scale_for(ex, em)); }
QS_HD double finish2(const Acc& lo, const Acc& hi, int ex, int em) { return finish2_s(lo, hi, scale_for(ex, em)); }

// Largest biased exponent of a set of doubles (exponent fields compared in
// place, on the high words).
QS_HD uint32_t expo_field(double x) {
  uint32_t hw, lw;
  qsdf::d2w(x, hw, lw);
  return hw & 0x7FF00000u;
}

}  // namespace qsfx
