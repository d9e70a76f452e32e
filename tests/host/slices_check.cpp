// Host check of the integer slicing used by the complex128 tensor-core kernel
// (qs_slices.cuh): digits reconstruct the rounded fixed-point value exactly,
// stay within their bounds and are exact in bf16; slice-product levels stay
// exact in FP32; the level recombination is exact; a full dot product of K
// terms stays within (K + 1) 2^-47 of the row-max x column-max scale with
// seven slices, (K + 1) 2^-54 with eight.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <random>
#include <vector>

#include "qs_slices.cuh"

static int failures = 0;
#define CHECK(cond, ...)                   \
  do {                                     \
    if (!(cond)) {                         \
      if (failures < 20) {                 \
        std::printf("FAIL: " __VA_ARGS__); \
        std::printf("\n");                 \
      }                                    \
      ++failures;                          \
    }                                      \
  } while (0)

static void words(double x, uint32_t& hw, uint32_t& lw) {
  uint64_t u;
  std::memcpy(&u, &x, 8);
  hw = (uint32_t)(u >> 32);
  lw = (uint32_t)u;
}

static int bexp(double x) {
  uint32_t hw, lw;
  words(x, hw, lw);
  return qsoz::biased_exp(hw);
}

// x 2^(48 - Emax) rounded half up, from long double arithmetic (exact here:
// the scaled value has at most 53 significant bits).
static long long ref_fixed(double x, int emax) {
  const long double y = std::ldexp((long double)x, 48 - (emax - 1023));
  return (long long)std::floor(y + 0.5L);
}

// bf16 bit pattern -> value
static float bf16_value(uint32_t h) { return qsdf::u2f((h & 0xFFFFu) << 16); }

static uint64_t fixed_of(int KS, double x, int emax) {
  uint32_t hw, lw;
  words(x, hw, lw);
  return KS == 8 ? qsoz::fixed_t8(hw, lw, emax) : qsoz::fixed_t(hw, lw, emax);
}

static int digit_of(int KS, uint64_t t, int s) { return KS == 8 ? qsoz::digit_t8(t, s) : qsoz::digit_t(t, s); }


// 9-12. Offset-packed digits: the packed bf16 halves decode to 192 + d_s; the
// top digit's float is d_0; combine_pairs agrees with the exact level sum; the
// accumulator started at P_L stays exact in FP32 for the extreme digits and
// K = 16, 32, 64, and ends at the level's bit pattern; whole dot products give
// the same integer as the float-digit path.
template <int KS>
static void check_packed(std::mt19937_64& rng) {
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  std::uniform_int_distribution<int> ex(-60, 10);
  const int floor_e = KS == 8 ? 58 : qsoz::kEmaxFloor;
  for (int it = 0; it < 1000000; ++it) {
    double xr = std::ldexp(u(rng), ex(rng)), xi = std::ldexp(u(rng), ex(rng));
    if (it % 97 == 0) xr = 0.0;
    if (it % 89 == 0) xi = -0.0;
    const int emax = std::max({floor_e, bexp(xr), bexp(xi)}) + (it % 3 == 0 ? 0 : (int)(rng() % 5));
    const uint64_t tr = fixed_of(KS, xr, emax), ti = fixed_of(KS, xi, emax);
    uint32_t w[KS], wf[KS];
    qsoz::packed_digits<KS>(tr, ti, w);
    qsoz::packed_digits_fast<KS>(tr, ti, wf);
    for (int s = 1; s < KS; ++s) {
      CHECK(w[s] == wf[s], "%d: byte-permute packing of digit %d", KS, s);
      CHECK(bf16_value(w[s]) == (float)(qsoz::kDigitOffset + digit_of(KS, tr, s)), "%d: packed re digit %d", KS, s);
      CHECK(bf16_value(w[s] >> 16) == (float)(qsoz::kDigitOffset + digit_of(KS, ti, s)), "%d: packed im digit %d",
            KS, s);
    }
    CHECK(qsoz::top_digit<KS>(tr) == (float)digit_of(KS, tr, 0), "%d: top digit", KS);
    CHECK((qsdf::f2u(qsoz::top_digit<KS>(ti)) & 0xFFFFu) == 0u, "%d: top digit not exact in bf16", KS);
  }

  // combine_pairs for both magic patterns (levels within the K <= 32 bound for
  // the preloaded magic, within the K = 64 bound for the added one)
  for (int pass = 0; pass < 2; ++pass) {
    const uint32_t mb = pass == 0 ? qsoz::kPreMagicBits : qsoz::kFaddMagicBits;
    const float magic = pass == 0 ? qsoz::kPreMagic : 12582912.0f;
    const int top = pass == 0 ? (KS == 8 ? 1310720 : 1179648) : (KS == 8 ? 2621440 : 2359296);   // level bounds
    std::uniform_int_distribution<int> lev(-top, top), lev0(-(1 << 20), 1 << 20);
    for (int it = 0; it < 1000000; ++it) {
      uint32_t bits[KS];
      __int128 sum = 0;
      for (int L = 0; L < KS; ++L) {
        const int t0 = L == 0 ? std::min(top, 1 << 20) : top;   // level 0: K 128 128 <= 2^20
        const int v = it < 3 ? (it == 0 ? t0 : (it == 1 ? -t0 : 0)) : (L == 0 ? lev0(rng) : lev(rng));
        bits[L] = qsdf::f2u((float)v + magic);
        CHECK(bits[L] == mb + (uint32_t)v, "%d: level %d bit pattern", KS, v);
        sum += (__int128)v * ((__int128)1 << (7 * (KS - 1 - L)));
      }
      const __int128 ref = KS == 8 ? (sum >> 8) : sum;
      CHECK((__int128)qsoz::combine_pairs<KS>(bits, mb) == ref, "%d: combine_pairs", KS);
      const long long got_u = pass == 0 ? qsoz::combine_pairs_u<KS, qsoz::kPreMagicBits>(bits)
                                        : qsoz::combine_pairs_u<KS, qsoz::kFaddMagicBits>(bits);
      CHECK((__int128)got_u == ref, "%d: combine_pairs_u (pass %d)", KS, pass);
    }
  }

  // the merged words of combine_pairs_u do not wrap for any levels within
  // the K <= 32 bound (preloaded magic) or the K <= 64 bound (added magic)
  for (int pass = 0; pass < 2; ++pass) {
    const long long top = pass == 0 ? (KS == 8 ? 1310720 : 1179648) : (KS == 8 ? 2621440 : 2359296);
    const long long off = (129ll * (pass == 0 ? qsoz::kPreMagicBits : qsoz::kFaddMagicBits)) & 0xFFFFFFFFll;
    for (long long hi : {-top, top})
      for (long long lo : {-top, top}) {
        const long long r = 128 * hi + lo + off;
        CHECK(r >= 0 && r < (1ll << 32), "%d: merged word wraps (pass %d)", KS, pass);
      }
  }

  // preloaded accumulators: every partial sum of P_L and the products, in any
  // order, stays an integer below 2^24 (bound over all terms), and the final
  // value has the level's bit pattern
  for (int K : {16, 32, 64}) {
    const float M = K <= 32 ? qsoz::kPreMagic : 0.0f;
    for (int it = 0; it < 4000; ++it) {
      int a[8][64], b[8][64];
      for (int s = 0; s < KS; ++s)
        for (int k = 0; k < K; ++k) {
          const int mag = s == 0 ? 128 : 64;
          const bool sa = it < 4 ? ((it >> (s == 0)) & 1) : (rng() & 1);
          const bool sb = it < 4 ? (it & 1) : (rng() & 1);
          a[s][k] = sa ? -mag : (s == 0 ? mag : 63);
          b[s][k] = sb ? -mag : (s == 0 ? mag : 63);
        }
      for (int L = 0; L < KS; ++L) {
        long long colsum = 0, abs_b = 0, abs_ab = 0, level = 0;
        std::vector<long long> terms;
        for (int t = 0; t <= L; ++t) {
          const int s = L - t;
          for (int k = 0; k < K; ++k) {
            const long long ap = s >= 1 ? qsoz::kDigitOffset + a[s][k] : a[s][k];
            terms.push_back(ap * b[t][k]);
            level += (long long)a[s][k] * b[t][k];
            abs_ab += std::llabs((long long)a[s][k] * b[t][k]);
            if (s >= 1) {
              colsum += b[t][k];
              abs_b += std::llabs(b[t][k]);
            }
          }
        }
        const long long P = (long long)M - qsoz::kDigitOffset * colsum;
        CHECK((long long)(float)P == P, "%d: P_L not exact (K = %d)", KS, K);
        // partial = M + sum_done a b - 192 sum_notdone b
        CHECK((long long)M + abs_ab + qsoz::kDigitOffset * abs_b < (1ll << 24), "%d: partial bound (K = %d, L = %d)",
              KS, K, L);
        CHECK((long long)M - abs_ab - qsoz::kDigitOffset * abs_b > -(1ll << 24), "%d: partial bound below", KS);
        std::shuffle(terms.begin(), terms.end(), rng);
        float acc = (float)P;
        long long ex_acc = P;
        for (long long tm : terms) {
          acc += (float)tm;
          ex_acc += tm;
          if ((long long)acc != ex_acc) break;
        }
        CHECK((long long)acc == ex_acc && ex_acc == (long long)M + level, "%d: preloaded level not exact", KS);
        const uint32_t bits = M != 0.0f ? qsdf::f2u(acc) : qsdf::f2u(acc + 12582912.0f);
        const uint32_t mb = M != 0.0f ? qsoz::kPreMagicBits : qsoz::kFaddMagicBits;
        CHECK(bits == mb + (uint32_t)level, "%d: level bit pattern (K = %d)", KS, K);
      }
    }
  }

  // the initialising MMA's column: three bf16-exact parts whose partial sums
  // stay below 2^24 (every start value |P| <= 2^24 - 2^21)
  for (int it = 0; it < 2000000; ++it) {
    const int P = it < 2 ? (it == 0 ? (1 << 24) - (1 << 21) : -(1 << 24) + (1 << 21))
                         : (int)(rng() % ((1u << 25) - (1u << 22))) - ((1 << 24) - (1 << 21));
    int pp[3];
    qsoz::split_start(P, pp);
    for (int k = 0; k < 3; ++k) {
      CHECK(std::abs(pp[k]) <= 256, "split part %d = %d", k, pp[k]);
      CHECK((qsdf::f2u((float)pp[k]) & 0xFFFFu) == 0u, "split part not exact in bf16");
    }
    CHECK(pp[0] + 256 * pp[1] + 65536 * pp[2] == P, "split of %d", P);
    CHECK(std::abs(65536 * pp[2]) < (1 << 24) && std::abs(65536 * pp[2] + 256 * pp[1]) < (1 << 24),
          "split partial sums of %d", P);
  }

  // whole dot products: offset-packed levels through combine_pairs equal the
  // float-digit levels through combine_levels / combine_levels8
  std::normal_distribution<double> gauss(0.0, 1.0);
  for (int it = 0; it < 20000; ++it) {
    const int K = 2 << (it % 5 + 1);  // 4 .. 64
    double a[64], b[64];
    std::uniform_int_distribution<int> es(it % 4 == 0 ? -40 : -3, 0);
    for (int k = 0; k < K; ++k) {
      a[k] = std::ldexp(gauss(rng), es(rng) - 15);
      b[k] = std::ldexp(gauss(rng), es(rng));
    }
    int ea = floor_e, eb = floor_e;
    for (int k = 0; k < K; ++k) {
      ea = std::max(ea, bexp(a[k]));
      eb = std::max(eb, bexp(b[k]));
    }
    long long lv[8] = {0}, colsum[8] = {0}, raw[8] = {0};
    for (int k = 0; k < K; ++k) {
      const uint64_t ta = fixed_of(KS, a[k], ea), tb = fixed_of(KS, b[k], eb);
      uint32_t w[KS];
      qsoz::packed_digits<KS>(ta, ta, w);
      for (int s = 0; s < KS; ++s)
        for (int t = 0; s + t < KS; ++t) {
          const long long ap = s == 0 ? (long long)qsoz::top_digit<KS>(ta) : (long long)bf16_value(w[s]);
          raw[s + t] += ap * digit_of(KS, tb, t);
          lv[s + t] += (long long)digit_of(KS, ta, s) * digit_of(KS, tb, t);
        }
      for (int t = 0; t < KS; ++t) colsum[t] += digit_of(KS, tb, t);
    }
    uint32_t bits_ref[8], bits_new[8];
    const bool pre = K <= 32;
    for (int L = 0; L < KS; ++L) {
      long long corr = 0;
      for (int t = 0; t < L; ++t) corr += colsum[t];
      const long long acc = (pre ? (long long)qsoz::kPreMagic : 0) - qsoz::kDigitOffset * corr + raw[L];
      bits_new[L] = pre ? qsdf::f2u((float)acc) : qsdf::f2u((float)acc + 12582912.0f);
      bits_ref[L] = qsdf::f2u((float)lv[L] + 12582912.0f);
    }
    const long long ref = KS == 8 ? qsoz::combine_levels8(bits_ref) : qsoz::combine_levels(bits_ref);
    const long long got = qsoz::combine_pairs<KS>(bits_new, pre ? qsoz::kPreMagicBits : qsoz::kFaddMagicBits);
    CHECK(got == ref, "%d: packed dot product %lld != %lld (K = %d)", KS, got, ref, K);
  }
}

int main() {
  std::mt19937_64 rng(2311015120ULL);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  std::uniform_int_distribution<int> ex(-60, 10);
  std::uniform_int_distribution<int> gap(0, 70);

  // 1. digits: exact reconstruction, bounds, float form exact in bf16
  for (int it = 0; it < 3000000; ++it) {
    double x = std::ldexp(u(rng), ex(rng));
    if (it % 97 == 0) x = 0.0;
    if (it % 101 == 0) x = -0.0;
    if (it % 103 == 0) x = std::ldexp(u(rng), -1040);   // subnormal: slices to zero
    if (it % 107 == 0) x = std::ldexp(u(rng), -990);    // below the floor of the grid
    int emax = (x == 0.0 ? 1000 : bexp(x)) + (it % 3 == 0 ? 0 : gap(rng) % (it % 5 == 0 ? 70 : 4));
    if (it % 7 == 0) emax = bexp(x);                    // value at the row maximum
    if (it % 11 == 0) emax += 1100;                     // shifts far above 63
    emax = std::max(emax, qsoz::kEmaxFloor);
    uint32_t hw, lw;
    words(x, hw, lw);
    const uint64_t w = qsoz::fixed_t(hw, lw, emax);
    long long v = 0;
    for (int s = 0; s < qsoz::kSlices; ++s) {
      const int d = qsoz::digit_t(w, s);
      if (s == 0)
        CHECK(d >= -128 && d <= 128, "d0 = %d", d);
      else
        CHECK(d >= -64 && d <= 63, "d%d = %d", s, d);
      v += (long long)d * (1ll << (42 - 7 * s));
    }
    const long long ref = ref_fixed(x, emax);
    CHECK(v == ref, "x = %.17g emax = %d: V = %lld, expected %lld", x, emax, v, ref);
    float f[qsoz::kSlices];
    qsoz::digit_floats_t(w, f);
    for (int s = 0; s < qsoz::kSlices; ++s) {
      CHECK(f[s] == (float)qsoz::digit_t(w, s), "float digit %d", s);
      CHECK((qsdf::f2u(f[s]) & 0xFFFFu) == 0u, "digit %d not exact in bf16", s);
    }
  }

  // 2. level sums of extreme digits stay below 2^22 and accumulate exactly in FP32
  for (int it = 0; it < 20000; ++it) {
    const int K = 64;
    int a[qsoz::kSlices][64], b[qsoz::kSlices][64];
    for (int s = 0; s < qsoz::kSlices; ++s)
      for (int k = 0; k < K; ++k) {
        const int mag = s == 0 ? 128 : 64;
        const bool sgn = it < 4 ? ((it >> (s == 0)) & 1) : (rng() & 1);
        a[s][k] = sgn ? -mag : (s == 0 ? mag : 63);
        b[s][k] = (it < 4 ? (it & 1) : (rng() & 1)) ? -mag : (s == 0 ? mag : 63);
      }
    for (int L = 0; L < qsoz::kSlices; ++L) {
      long long exact = 0;
      float acc = 0.0f;
      for (int s = 0; s <= L; ++s)
        for (int k = 0; k < K; ++k) {
          const long long p = (long long)a[s][k] * b[L - s][k];
          exact += p;
          acc += (float)p;
        }
      CHECK(std::llabs(exact) < (1ll << 22), "level %d = %lld", L, exact);
      CHECK((long long)acc == exact, "level %d not exact in FP32", L);
    }
  }

  // 3. recombination of the level bit patterns
  // (level 0 is below 2^20: K * 128 * 128 with K <= 64)
  std::uniform_int_distribution<int> lev(-(1 << 22) + 1, (1 << 22) - 1);
  std::uniform_int_distribution<int> lev0(-(1 << 20), 1 << 20);
  for (int it = 0; it < 2000000; ++it) {
    uint32_t bits[qsoz::kSlices];
    __int128 ref = 0;
    for (int L = 0; L < qsoz::kSlices; ++L) {
      const int top = L == 0 ? (1 << 20) : (1 << 22) - 1;
      const int v = it < 3 ? (it == 0 ? top : (it == 1 ? -top : 0)) : (L == 0 ? lev0(rng) : lev(rng));
      bits[L] = qsdf::f2u((float)v + 12582912.0f);
      ref += (__int128)v * ((__int128)1 << (7 * (6 - L)));
    }
    const long long got = qsoz::combine_levels(bits);
    CHECK((__int128)got == ref, "combine %lld", got);
  }

  // 4. full complex dot products through digits, levels and recombination
  std::normal_distribution<double> gauss(0.0, 1.0);
  double worst = 0.0;
  for (int it = 0; it < 20000; ++it) {
    const int K = 2 << (it % 5 + 1);  // 4 .. 64
    double a[64], b[64];
    const int spread = it % 4 == 0 ? 40 : 3;
    std::uniform_int_distribution<int> es(-spread, 0);
    for (int k = 0; k < K; ++k) {
      a[k] = std::ldexp(gauss(rng), es(rng) - 15);
      b[k] = std::ldexp(gauss(rng), es(rng));
    }
    int ea = qsoz::kEmaxFloor, eb = qsoz::kEmaxFloor;
    for (int k = 0; k < K; ++k) {
      ea = std::max(ea, bexp(a[k]));
      eb = std::max(eb, bexp(b[k]));
    }
    long long lv[qsoz::kSlices] = {0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < K; ++k) {
      uint32_t h1, l1, h2, l2;
      words(a[k], h1, l1);
      words(b[k], h2, l2);
      const uint64_t wa = qsoz::fixed_t(h1, l1, ea), wb = qsoz::fixed_t(h2, l2, eb);
      for (int s = 0; s < qsoz::kSlices; ++s)
        for (int t = 0; s + t < qsoz::kSlices; ++t) lv[s + t] += (long long)qsoz::digit_t(wa, s) * qsoz::digit_t(wb, t);
    }
    uint32_t bits[qsoz::kSlices];
    for (int L = 0; L < qsoz::kSlices; ++L) bits[L] = qsdf::f2u((float)lv[L] + 12582912.0f);
    const long long acc = qsoz::combine_levels(bits);
    const long double got = std::ldexp((long double)acc, (ea - 1023) + (eb - 1023) - 54);
    long double exact = 0;
    for (int k = 0; k < K; ++k) exact += (long double)a[k] * b[k];
    const long double scale = std::ldexp(1.0L, (ea - 1023) + (eb - 1023) + 1);
    const double rel = (double)(std::fabs(got - exact) / scale);
    worst = std::max(worst, rel);
    // each term carries at most 2^-47 of the scale (two operand roundings of
    // 2^-49 relative to the maxima), and the dropped levels add below 2^-47
    CHECK(rel < (K + 1) * std::ldexp(1.0, -47), "dot product error %.3g of the scale (K = %d)", rel, K);
  }
  std::printf("worst dot-product error / (row max * column max) = %.3g (2^%.1f)\n", worst, std::log2(worst));

  // ---- eight slices (qsoz::*8: 56-bit operands) ----
  // 5. digits: exact reconstruction of x 2^(55 - Emax) rounded half up, bounds, bf16
  constexpr int kS8 = qsoz::kSlices8;
  constexpr int kFloor8 = 58;
  for (int it = 0; it < 3000000; ++it) {
    double x = std::ldexp(u(rng), ex(rng));
    if (it % 97 == 0) x = 0.0;
    if (it % 101 == 0) x = -0.0;
    if (it % 103 == 0) x = std::ldexp(u(rng), -1040);
    if (it % 107 == 0) x = std::ldexp(u(rng), -990);
    int emax = (x == 0.0 ? 1000 : bexp(x)) + (it % 3 == 0 ? 0 : gap(rng) % (it % 5 == 0 ? 70 : 4));
    if (it % 7 == 0) emax = bexp(x);
    if (it % 11 == 0) emax += 1100;
    emax = std::max(emax, kFloor8);
    uint32_t hw, lw;
    words(x, hw, lw);
    const uint64_t w = qsoz::fixed_t8(hw, lw, emax);
    long long v = 0;
    for (int s = 0; s < kS8; ++s) {
      const int d = qsoz::digit_t8(w, s);
      if (s == 0)
        CHECK(d >= -128 && d <= 128, "8: d0 = %d", d);
      else
        CHECK(d >= -64 && d <= 63, "8: d%d = %d", s, d);
      v += (long long)d * (1ll << (49 - 7 * s));
    }
    const long double y = std::ldexp((long double)x, 55 - (emax - 1023));
    const long long ref = (long long)std::floor(y + 0.5L);
    CHECK(v == ref, "8: x = %.17g emax = %d: V = %lld, expected %lld", x, emax, v, ref);
    float f[kS8];
    qsoz::digit_floats_t8(w, f);
    for (int s = 0; s < kS8; ++s) {
      CHECK(f[s] == (float)qsoz::digit_t8(w, s), "8: float digit %d", s);
      CHECK((qsdf::f2u(f[s]) & 0xFFFFu) == 0u, "8: digit %d not exact in bf16", s);
    }
  }

  // 6. levels 0..7 of extreme digits stay below 2^22 and are exact in FP32
  for (int it = 0; it < 20000; ++it) {
    const int K = 64;
    int a[kS8][64], b[kS8][64];
    for (int s = 0; s < kS8; ++s)
      for (int k = 0; k < K; ++k) {
        const int mag = s == 0 ? 128 : 64;
        const bool sgn = it < 4 ? ((it >> (s == 0)) & 1) : (rng() & 1);
        a[s][k] = sgn ? -mag : (s == 0 ? mag : 63);
        b[s][k] = (it < 4 ? (it & 1) : (rng() & 1)) ? -mag : (s == 0 ? mag : 63);
      }
    for (int L = 0; L < kS8; ++L) {
      long long exact = 0;
      float acc = 0.0f;
      for (int s = 0; s <= L; ++s)
        for (int k = 0; k < K; ++k) {
          const long long p = (long long)a[s][k] * b[L - s][k];
          exact += p;
          acc += (float)p;
        }
      CHECK(std::llabs(exact) < (1ll << 22), "8: level %d = %lld", L, exact);
      CHECK((long long)acc == exact, "8: level %d not exact in FP32", L);
    }
  }

  // 7. recombination: floor(sum_L level_L 2^(7(7-L)) / 2^8), whenever the true
  // value fits in 63 bits (levels up to 2.5 2^20, level 0 up to 2^20)
  std::uniform_int_distribution<int> lev8(-(5 << 19), 5 << 19);
  for (int it = 0; it < 2000000; ++it) {
    uint32_t bits[8];
    __int128 sum = 0;
    for (int L = 0; L < kS8; ++L) {
      const int top = L == 0 ? (1 << 20) : (5 << 19);
      const int v = it < 3 ? (it == 0 ? top : (it == 1 ? -top : 0)) : (L == 0 ? lev0(rng) : lev8(rng));
      bits[L] = qsdf::f2u((float)v + 12582912.0f);
      sum += (__int128)v * ((__int128)1 << (7 * (7 - L)));
    }
    // floor division by 2^8
    __int128 ref = sum >> 8;
    const long long got = qsoz::combine_levels8(bits);
    CHECK((__int128)got == ref, "8: combine %lld", got);
  }

  // 8. full dot products through eight digits: within (K + 1) 2^-54 of the scale
  double worst8 = 0.0;
  for (int it = 0; it < 20000; ++it) {
    const int K = 2 << (it % 5 + 1);  // 4 .. 64
    double a[64], b[64];
    const int spread = it % 4 == 0 ? 40 : 3;
    std::uniform_int_distribution<int> es(-spread, 0);
    for (int k = 0; k < K; ++k) {
      a[k] = std::ldexp(gauss(rng), es(rng) - 15);
      b[k] = std::ldexp(gauss(rng), es(rng));
    }
    int ea = kFloor8, eb = kFloor8;
    for (int k = 0; k < K; ++k) {
      ea = std::max(ea, bexp(a[k]));
      eb = std::max(eb, bexp(b[k]));
    }
    long long lv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < K; ++k) {
      uint32_t h1, l1, h2, l2;
      words(a[k], h1, l1);
      words(b[k], h2, l2);
      const uint64_t wa = qsoz::fixed_t8(h1, l1, ea), wb = qsoz::fixed_t8(h2, l2, eb);
      for (int s = 0; s < kS8; ++s)
        for (int t = 0; s + t < kS8; ++t) lv[s + t] += (long long)qsoz::digit_t8(wa, s) * qsoz::digit_t8(wb, t);
    }
    uint32_t bits[8];
    for (int L = 0; L < kS8; ++L) bits[L] = qsdf::f2u((float)lv[L] + 12582912.0f);
    const long long acc = qsoz::combine_levels8(bits);
    const long double got = std::ldexp((long double)acc, (ea - 1023) + (eb - 1023) - 53);
    long double exact = 0;
    for (int k = 0; k < K; ++k) exact += (long double)a[k] * b[k];
    const long double scale = std::ldexp(1.0L, (ea - 1023) + (eb - 1023) + 1);
    const double rel = (double)(std::fabs(got - exact) / scale);
    worst8 = std::max(worst8, rel);
    CHECK(rel < (K + 1) * std::ldexp(1.0, -54), "8: dot product error %.3g of the scale (K = %d)", rel, K);
  }
  std::printf("eight slices: worst dot-product error / (row max * column max) = %.3g (2^%.1f)\n", worst8,
              std::log2(worst8));

  // ---- offset-packed amplitude digits (both slice counts) ----
  check_packed<7>(rng);
  check_packed<8>(rng);

  std::printf("ok (%d failures)\n", failures);
  return failures ? 1 : 0;
}
