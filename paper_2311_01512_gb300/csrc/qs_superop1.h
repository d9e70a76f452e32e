// Superoperator of a one-qubit Kraus map, formed on the host (no CUDA
// dependency, so the host check tests/host/superop1_check.cpp compiles it
// with g++ alone).
#pragma once

namespace qsh {

// sum_m conj(K_m) (x) K_m of one-qubit operators K_m (row-major 2x2, re/im
// interleaved) as a 4x4 matrix (Sec. "Kraus map"): row r = 2 i + k, column
// c = 2 j + l, entry sum_m conj(K_m[i][j]) K_m[k][l]; index bit 0 acts on the
// ket qubit t, bit 1 on the bra qubit t + N.  The same entries as the device
// superoperator kernel; the library makes the block fixed-point constants of
// a one-pass Kraus map from it.  sup: 32 doubles (16 complex, row-major).
inline void superop1(const double* kraus, int num_ops, double* sup) {
  for (int e = 0; e < 32; ++e) sup[e] = 0.0;
  for (int m = 0; m < num_ops; ++m) {
    const double* K = kraus + 8 * m;
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) {
        const int a = 2 * (r >> 1) + (c >> 1), b = 2 * (r & 1) + (c & 1);
        const double ar = K[2 * a], ai = -K[2 * a + 1], br = K[2 * b], bi = K[2 * b + 1];
        sup[2 * (4 * r + c)] += ar * br - ai * bi;
        sup[2 * (4 * r + c) + 1] += ar * bi + ai * br;
      }
  }
}

}  // namespace qsh
