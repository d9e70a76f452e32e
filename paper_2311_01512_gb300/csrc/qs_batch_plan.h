// Host-only parts of the batched engine that need no GPU: the segment
// planner (cache blocking of states larger than shared memory) and the
// superoperators that density-matrix operations are lowered to.  Used by
// qs_batch.cpp and checked on the CPU by tests/host/batch_plan_check.cpp.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "qs_internal.h"

namespace qsbatch {

inline int popc32(uint32_t x) {
  int n = 0;
  for (; x; x &= x - 1) ++n;
  return n;
}

// qubits an operation pairs amplitudes across
inline uint32_t pairing_mask(const qsk::BatchOp& op) {
  if (op.kind == 0) {
    uint32_t m = 0;
    for (int q = 0; q < op.n; ++q) m |= 1u << op.t[q];
    return m;
  }
  return op.kind == 2 ? op.xy : 0u;
}

// position of qubit t among the tile qubits, -1 if it is not one
inline int local_pos(uint32_t qmask, int t) {
  return ((qmask >> t) & 1u) ? popc32(qmask & ((1u << t) - 1u)) : -1;
}

inline qsk::BatchXlat translate(const qsk::BatchOp& op, uint32_t qmask) {
  qsk::BatchXlat x{};
  for (int q = 0; q < 4; ++q) x.lt[q] = -1;
  if (op.kind == 0) {
    std::vector<int> lins;
    for (int q = 0; q < op.n; ++q) {
      x.lt[q] = (int8_t)local_pos(qmask, op.t[q]);
      lins.push_back(x.lt[q]);
    }
    for (int c = 0; c < 32; ++c) {
      if (!((op.ctrl >> c) & 1u)) continue;
      const int p = local_pos(qmask, c);
      if (p >= 0) {
        x.lctrl |= 1u << p;
        lins.push_back(p);
      } else {
        x.fctrl |= 1u << c;
      }
    }
    std::sort(lins.begin(), lins.end());
    x.nlins = (int)lins.size();
    for (int i = 0; i < x.nlins; ++i) x.lins[i] = (int8_t)lins[i];
  } else if (op.kind == 1) {
    for (int q = 0; q < op.n; ++q) x.lt[q] = (int8_t)local_pos(qmask, op.t[q]);
  } else {
    for (int b = 0; b < 32; ++b) {
      const int p = local_pos(qmask, b);
      if ((op.xy >> b) & 1u) x.lxy |= 1u << p;       // every flip qubit is a tile qubit
      if ((op.yz >> b) & 1u) {
        if (p >= 0)
          x.lyz |= 1u << p;
        else
          x.fyz |= 1u << b;
      }
    }
    x.lh = (int8_t)(op.xy ? local_pos(qmask, op.h) : 0);
  }
  return x;
}

// Segments of every state larger than 2^L amplitudes (states[s].first_seg and
// nsegs are set; xlat gets one entry per operation).  Greedy: an operation
// joins the open segment while the union of pairing qubits and the five
// lowest qubits stays within L; an operation that alone exceeds it runs in
// global memory (a segment with L = 0).  The tile qubits are that union,
// filled up with the lowest remaining qubits.
inline void build_segments(int L, const std::vector<int>& nq, std::vector<qsk::BatchState>& states,
                           const std::vector<qsk::BatchOp>& ops, std::vector<qsk::BatchSeg>& segs,
                           std::vector<qsk::BatchXlat>& xlat) {
  segs.clear();
  xlat.assign(ops.size(), qsk::BatchXlat{});
  for (size_t s = 0; s < states.size(); ++s) {
    qsk::BatchState& st = states[s];
    st.first_seg = (int)segs.size();
    st.nsegs = 0;
    if (nq[s] <= L) continue;
    const uint32_t low = (1u << std::min(5, nq[s])) - 1u;
    auto emit = [&](int first, int n, uint32_t U, bool tiled) {
      qsk::BatchSeg g{};
      g.first_op = first;
      g.nops = n;
      g.L = tiled ? L : 0;
      if (tiled) {
        uint32_t Q = low | U;
        for (int b = 0; popc32(Q) < L; ++b) Q |= 1u << b;
        for (int b = 0, i = 0; b < 32; ++b)
          if ((Q >> b) & 1u) g.q[i++] = (int8_t)b;
        for (int k = first; k < first + n; ++k) xlat[k] = translate(ops[k], Q);
      }
      segs.push_back(g);
    };
    int k0 = st.first_op, cnt = 0;
    uint32_t U = 0;
    for (int k = st.first_op; k < st.first_op + st.nops; ++k) {
      const uint32_t pm = pairing_mask(ops[k]);
      if (popc32(low | pm) > L) {
        if (cnt) emit(k0, cnt, U, true);
        emit(k, 1, 0u, false);
        k0 = k + 1;
        cnt = 0;
        U = 0;
        continue;
      }
      if (popc32(low | U | pm) > L) {
        emit(k0, cnt, U, true);
        k0 = k;
        cnt = 0;
        U = 0;
      }
      U |= pm;
      ++cnt;
    }
    if (cnt) emit(k0, cnt, U, true);
    st.nsegs = (int)segs.size() - st.first_seg;
  }
}

// ---- superoperators on the Choi vector (Sec. "Kraus map") -------------------
// Member m of a group has bit q of m on the q-th of the positions (t, t + N)
// (one qubit) or (t1, t2, t1 + N, t2 + N) (two qubits); S (row-major, d x d)
// gives new beta_m = sum_k S[m][k] beta_k.

// S = sum_m conj(K_m) (x) K_m, complex (re, im interleaved): K on the ket bits
// t (the low n bits of the member index), conj(K) on the bra bits t + N.
inline std::vector<double> kraus_superop(int n, const double* kraus, int num_ops) {
  const int d = 1 << n, dd = d * d;
  std::vector<double> m((size_t)2 * dd * dd, 0.0);
  for (int k = 0; k < num_ops; ++k) {
    const double* K = kraus + (size_t)2 * d * d * k;
    for (int ih = 0; ih < d; ++ih)
      for (int il = 0; il < d; ++il)
        for (int jh = 0; jh < d; ++jh)
          for (int jl = 0; jl < d; ++jl) {
            const double ar = K[2 * (ih * d + jh)], ai = -K[2 * (ih * d + jh) + 1];   // conj(K[ih][jh])
            const double br = K[2 * (il * d + jl)], bi = K[2 * (il * d + jl) + 1];
            const size_t e = (size_t)(ih * d + il) * dd + (jh * d + jl);
            m[2 * e] += ar * br - ai * bi;
            m[2 * e + 1] += ar * bi + ai * br;
          }
  }
  return m;
}

// One-qubit channels in the paper's Choi-vector form (real 4 x 4): members 00
// and 11 mix as f0 self + f1 other, 01 and 10 as f2 self + f3 other.
inline std::vector<double> channel1_superop(double f0, double f1, double f2, double f3) {
  std::vector<double> S(16, 0.0);
  S[0 * 4 + 0] = f0;
  S[0 * 4 + 3] = f1;
  S[3 * 4 + 3] = f0;
  S[3 * 4 + 0] = f1;
  S[1 * 4 + 1] = f2;
  S[1 * 4 + 2] = f3;
  S[2 * 4 + 2] = f2;
  S[2 * 4 + 1] = f3;
  return S;
}

// Amplitude damping (Sec. "Damping channel"): 00 -> 00 + p 11; 01, 10 scale
// by sqrt(1 - p); 11 by 1 - p.
inline std::vector<double> damping_superop(double p) {
  std::vector<double> S(16, 0.0);
  S[0 * 4 + 0] = 1.0;
  S[0 * 4 + 3] = p;
  S[1 * 4 + 1] = std::sqrt(1.0 - p);
  S[2 * 4 + 2] = std::sqrt(1.0 - p);
  S[3 * 4 + 3] = 1.0 - p;
  return S;
}

// Two-qubit dephasing and depolarising (Sec. "Dephasing channel",
// "Depolarising channel", two-qubit update rules), real 16 x 16.
inline std::vector<double> channel2_superop(bool depol, double p) {
  std::vector<double> S(256, 0.0);
  for (int m = 0; m < 16; ++m) {
    const bool same1 = ((m >> 0) & 1) == ((m >> 2) & 1), same2 = ((m >> 1) & 1) == ((m >> 3) & 1);
    if (!depol) {
      S[m * 16 + m] = (same1 && same2) ? 1.0 : 1.0 - 4.0 * p / 3.0;
    } else if (same1 && same2) {
      S[m * 16 + m] = 1.0 - 4.0 * p / 5.0;
      for (int f : {0x5, 0xA, 0xF}) S[m * 16 + (m ^ f)] = 4.0 * p / 15.0;   // flip t1 pair, t2 pair, both
    } else {
      S[m * 16 + m] = 1.0 - 16.0 * p / 15.0;
    }
  }
  return S;
}

}  // namespace qsbatch
