// Host check of the statevector expectation's tile order (make_tile_order and
// ordered_tile in qs_internal.h): for random Pauli sums the map from virtual
// position to tile is a bijection, and every term pairs each tile with a tile
// of the same block of 2^r consecutive positions (one coset of the span of
// the flip masks' tile bits), which is what lets the blocks that walk the
// positions in order find a tile's partners in L2.
#include <cstdio>
#include <random>
#include <vector>

#include "qs_internal.h"

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

int main() {
  std::mt19937_64 rng(2311015124ULL);
  for (int it = 0; it < 400; ++it) {
    const int nq = 11 + (int)(rng() % 13);                 // 11 .. 23 qubits: 2 .. 8192 tiles
    const int ntiles_bits = nq - qsk::kExpecTileBits;
    const uint64_t ntiles = 1ull << ntiles_bits;
    const int nterms = 1 + (int)(rng() % (it % 3 == 0 ? 40 : 8));
    std::vector<qsk::PauliTerm> terms(nterms);
    for (auto& t : terms) {
      t = qsk::PauliTerm{};
      t.xy = rng() & ((1ull << nq) - 1);
      if (it % 5 == 0) t.xy &= (1ull << qsk::kExpecTileBits) - 1;   // flips inside a tile only
      if (it % 7 == 0) t.xy = terms[0].xy ^ (terms.size() > 1 ? terms[1].xy : 0);   // dependent masks
    }
    const qsk::TileOrder o = qsk::make_tile_order(terms.data(), nterms);
    CHECK(o.r >= 0 && o.r <= ntiles_bits, "rank %d of %d tile bits", o.r, ntiles_bits);
    std::vector<int64_t> pos(ntiles, -1);
    for (uint64_t v = 0; v < ntiles; ++v) {
      const uint64_t t = qsk::ordered_tile(v, o);
      CHECK(t < ntiles, "tile %llu out of range", (unsigned long long)t);
      if (t < ntiles) {
        CHECK(pos[t] < 0, "tile %llu visited twice", (unsigned long long)t);
        pos[t] = (int64_t)v;
      }
    }
    for (uint64_t v = 0; v < ntiles && failures == 0; ++v) {
      const uint64_t t = qsk::ordered_tile(v, o);
      for (const auto& term : terms) {
        const uint64_t partner = t ^ (term.xy >> qsk::kExpecTileBits);
        CHECK(partner < ntiles && ((uint64_t)pos[partner] >> o.r) == (v >> o.r),
              "partner of tile %llu outside its block (r = %d)", (unsigned long long)t, o.r);
      }
    }
  }
  std::printf("ok (%d failures)\n", failures);
  return failures ? 1 : 0;
}
