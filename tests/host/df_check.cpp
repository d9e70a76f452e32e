// Host check of the double-float split/join/dot logic in qs_df.cuh (the same
// integer and FP32 operations the kernels run).  Prints failures and exits 1.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <random>

#include "qs_df.cuh"

using qsdf::df;

static int failures = 0;
static void fail(const char* what, double a, double b) {
  if (failures++ < 20) std::printf("FAIL %s: %.17g vs %.17g\n", what, a, b);
}

int main() {
  std::mt19937_64 rng(2311015120ULL);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  std::uniform_int_distribution<int> ex(-100, 100);
  // 1. split keeps 47 bits: hi + lo within 2^-47 |x|, hi is the truncation to 24 bits
  long double bias = 0;
  long nbias = 0;
  for (int i = 0; i < 2000000; ++i) {
    const double x = std::ldexp(u(rng), ex(rng));
    const df s = qsdf::split(x);
    // bound: 2^-47 relative, or 2^-103 absolute below 2^-80
    const double tol = std::fmax(std::ldexp(std::fabs(x), -47), std::ldexp(1.0, -103));
    const double back = (double)s.h + (double)s.l;
    if (std::fabs(back - x) > tol) fail("split", back, x);
    if (std::fabs(x) >= std::ldexp(1.0, -103) &&
        (double)s.h != std::ldexp(std::trunc(std::ldexp(x, 23 - std::ilogb(x))), std::ilogb(x) - 23))
      fail("split hi", s.h, x);
    // 2. join(split(x)) recovers x to the same bound
    const double j = qsdf::join(s);
    if (std::fabs(j - x) > tol) fail("join(split)", j, x);
    if (std::fabs(x) >= std::ldexp(1.0, -80)) {
      bias += (long double)(j - x) / std::fabs(x);
      ++nbias;
    }
  }
  // 2b. no systematic bias toward zero: the mean relative error of the round
  // trip is far below its per-sample bound
  if (std::fabs((double)(bias / nbias)) > std::ldexp(1.0, -56)) fail("round-trip bias", (double)(bias / nbias), 0.0);
  // 3. join of normalised pairs from TwoSum equals IEEE round-to-nearest-even of h + l
  for (int i = 0; i < 2000000; ++i) {
    const int e = ex(rng) / 2;
    const float a = (float)std::ldexp(u(rng), e), b = (float)std::ldexp(u(rng), e - (i % 40));
    const float h = a + b;
    const float bb = h - a;
    const float l = (a - (h - bb)) + (b - bb);
    const double want = (double)a + (double)b;          // IEEE round-to-nearest-even
    const double got = qsdf::join(df{h, l});
    if (got != want) fail("join pair", got, want);
  }
  // powers of two with an opposite-sign tail (the borrow case) and zeros
  {
    const float hs[] = {1.0f, -0.5f, 0.25f, -1024.0f, 1.0f};
    const float ls[] = {-std::ldexp(1.0f, -30), std::ldexp(1.0f, -31), -std::ldexp(3.0f, -28), 1e-5f, 0.0f};
    for (int i = 0; i < 5; ++i) {
      const double want = (double)hs[i] + (double)ls[i];
      const double got = qsdf::join(df{hs[i], ls[i]});
      if (got != want) fail("join pow2", got, want);
    }
    if (qsdf::join(df{0.0f, 0.0f}) != 0.0) fail("join zero", qsdf::join(df{0.0f, 0.0f}), 0.0);
    const df z = qsdf::split(0.0), nz = qsdf::split(-0.0), tiny = qsdf::split(1e-40), sub = qsdf::split(5e-320);
    if (z.h != 0 || z.l != 0 || nz.h != 0 || tiny.h != 0 || tiny.l != 0 || sub.h != 0) fail("split zero", z.h, 0);
    const df at = qsdf::split(std::ldexp(1.5, -102));
    if ((double)at.h + (double)at.l != std::ldexp(1.5, -102)) fail("split 2^-102", at.h, 0);
  }
  // 3b. to_double is exact for normal floats and signed zeros; FP32 subnormals
  // land within 2^-126 (below the documented range)
  for (int i = 0; i < 1000000; ++i) {
    const float f = (float)std::ldexp(u(rng), ex(rng));
    const double got = qsdf::to_double(f);
    if (std::fabs(f) >= std::ldexp(1.0f, -126)) {
      if (got != (double)f) fail("to_double", got, (double)f);
    } else if (std::fabs(got - (double)f) > std::ldexp(1.0, -126)) {
      fail("to_double subnormal", got, (double)f);
    }
  }
  for (uint32_t bits : {0x00000001u, 0x007FFFFFu, 0x80000001u, 0x807FFFFFu, 0x00400000u}) {
    float f;
    std::memcpy(&f, &bits, 4);
    if (std::fabs(qsdf::to_double(f)) > std::ldexp(1.0, -126)) fail("to_double subnormal edge", qsdf::to_double(f), 0);
  }
  if (qsdf::to_double(0.0f) != 0.0 || std::signbit(qsdf::to_double(0.0f))) fail("to_double +0", 0, 0);
  if (qsdf::to_double(-0.0f) != 0.0 || !std::signbit(qsdf::to_double(-0.0f))) fail("to_double -0", 0, 0);
  for (float f : {1.0f, -1.0f, 3.4028235e38f, -3.4028235e38f, 1.17549435e-38f, -1.17549435e-38f})
    if (qsdf::to_double(f) != (double)f) fail("to_double edge", qsdf::to_double(f), (double)f);
  // 4. dot products of length 2..64 against long double: error <= 16 * 2^-46 * sum |c v|
  for (int i = 0; i < 300000; ++i) {
    const int len = 2 + (i % 63);
    double c[64], v[64];
    long double ref = 0, mag = 0;
    for (int k = 0; k < len; ++k) {
      c[k] = u(rng);
      v[k] = std::ldexp(u(rng), -(i % 30));
      ref += (long double)c[k] * v[k];
      mag += std::fabs((long double)c[k] * v[k]);
    }
    qsdf::dot_acc a = qsdf::dot_first(qsdf::split_const(c[0]), qsdf::split(v[0]));
    for (int k = 1; k < len; ++k) qsdf::dot_add(a, qsdf::split_const(c[k]), qsdf::split(v[k]));
    const double got = qsdf::join(qsdf::dot_result(a));
    if (std::fabs((long double)got - ref) > 16.0L * std::ldexp(1.0L, -46) * mag) fail("dot", got, (double)ref);
    const double fin = qsdf::finish(a);
    if (std::fabs((long double)fin - ref) > 16.0L * std::ldexp(1.0L, -46) * mag) fail("dot finish", fin, (double)ref);
  }
  std::printf("%s (%d failures)\n", failures ? "FAILED" : "ok", failures);
  return failures ? 1 : 0;
}
