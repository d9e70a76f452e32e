// Host program for the one-qubit superoperator the library forms on the host
// (paper_2311_01512_gb300/csrc/qs_superop1.h): reads Kraus sets from stdin and
// prints the 4x4 superoperator, so the Python test can compare it with the
// oracle's superoperator and Kraus map.
//
// Input, one case per line: m followed by 8 m hex doubles (K_0 .. K_{m-1},
// each row-major 2x2, re/im interleaved).  Output, one line per case: the 32
// doubles of the superoperator in hex.
#include <cstdio>

#include "qs_superop1.h"

int main() {
  int m;
  while (std::scanf("%d", &m) == 1) {
    if (m < 1 || m > 16) return 2;
    double k[16 * 8], sup[32];
    for (int e = 0; e < 8 * m; ++e)
      if (std::scanf("%la", &k[e]) != 1) return 2;
    qsh::superop1(k, m, sup);
    for (int e = 0; e < 32; ++e) std::printf(e ? " %a" : "%a", sup[e]);
    std::printf("\n");
  }
  return 0;
}
