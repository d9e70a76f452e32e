// Host program for the block fixed-point arithmetic (qs_fx.cuh): reads dot
// products from stdin and prints what the kernels compute for them, so that
// the Python test can compare with exact rational arithmetic.
//
// Input, one case per line (64-bit patterns of doubles in hex):
//   K x_0 .. x_{K-1} m_0 .. m_{K-1}      (1 <= K <= 8)
// Output, one line per case:
//   y  M_0 .. M_{K-1}
// with y = sum_k x_k m_k in block fixed point (the x_k share their largest
// exponent, the m_k theirs, as the kernels and the C-ABI group them; terms
// 4..7 in a second accumulator, as the two-target gate sums them), and
// M_k = the 60-bit fixed-point constant of m_k (h 2^30 + l, decimal).
#include <cinttypes>
#include <cstdio>
#include <cstring>

#include "qs_fx.cuh"

static double from_bits(uint64_t u) {
  double x;
  std::memcpy(&x, &u, 8);
  return x;
}
static uint64_t to_bits(double x) {
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return u;
}

int main() {
  int K;
  while (std::scanf("%d", &K) == 1) {
    if (K < 1 || K > 8) return 2;
    double x[8], m[8];
    for (int k = 0; k < K; ++k) {
      uint64_t u;
      if (std::scanf("%" SCNx64, &u) != 1) return 2;
      x[k] = from_bits(u);
    }
    for (int k = 0; k < K; ++k) {
      uint64_t u;
      if (std::scanf("%" SCNx64, &u) != 1) return 2;
      m[k] = from_bits(u);
    }
    int ex = 0, em = 0;
    for (int k = 0; k < K; ++k) {
      ex = ex > qsfx::expo_of(x[k]) ? ex : qsfx::expo_of(x[k]);
      em = em > qsfx::expo_of(m[k]) ? em : qsfx::expo_of(m[k]);
    }
    qsfx::Acc acc[2] = {qsfx::acc_zero(), qsfx::acc_zero()};
    qsfx::Part mp[8];
    for (int k = 0; k < K; ++k) {
      mp[k] = qsfx::fixed_const(m[k], em);
      qsfx::mac(acc[k >> 2], qsfx::fixed_d(x[k], ex), mp[k]);
    }
    const double y = K <= 4 ? qsfx::finish(acc[0], ex, em) : qsfx::finish2(acc[0], acc[1], ex, em);
    std::printf("%016" PRIx64, to_bits(y));
    for (int k = 0; k < K; ++k) std::printf(" %" PRId64, (int64_t)mp[k].h * (1ll << 30) + mp[k].l);
    std::printf("\n");
  }
  return 0;
}
