// Host check of the batched engine's host-only parts (qs_batch_plan.h).
//
// Reads commands from standard input, one per line:
//   plan                      random batches through the segment planner; its
//                             invariants are checked here and the line
//                             "plan ok (F failures)" is printed
//   c1 f0 f1 f2 f3            one-qubit channel superoperator (16 reals)
//   damp p                    damping superoperator (16 reals)
//   c2 depol p                two-qubit channel superoperator (256 reals)
//   kraus n m v...            superoperator of m Kraus operators on n qubits
//                             (2 * m * 4^n input reals, 2 * 16^n output reals)
// Superoperators are printed on one line each, for the caller to compare with
// the oracle's channels.
#include <cstdio>
#include <iostream>
#include <random>
#include <sstream>
#include <string>
#include <vector>

#include "qs_batch_plan.h"

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

static void print(const std::vector<double>& v) {
  for (size_t i = 0; i < v.size(); ++i) std::printf(i ? " %.17g" : "%.17g", v[i]);
  std::printf("\n");
}

static void check_plan() {
  std::mt19937 rng(20231101);
  for (int it = 0; it < 400; ++it) {
    const int L = 8 + (int)(rng() % 7);                 // 8 .. 14
    const int S = 1 + (int)(rng() % 6);
    std::vector<int> nq;
    std::vector<qsk::BatchState> states(S);
    std::vector<qsk::BatchOp> ops;
    for (int s = 0; s < S; ++s) {
      nq.push_back(5 + (int)(rng() % 20));              // 5 .. 24
      states[s].nq = nq[s];
      states[s].first_op = (int)ops.size();
      const int n_ops = (int)(rng() % 40);
      for (int k = 0; k < n_ops; ++k) {
        qsk::BatchOp op{};
        op.kind = (int)(rng() % 3);
        std::vector<int> perm(nq[s]);
        for (int q = 0; q < nq[s]; ++q) perm[q] = q;
        std::shuffle(perm.begin(), perm.end(), rng);
        if (op.kind == 0) {
          op.n = 1 + (int)(rng() % 4);
          const int nc = (int)(rng() % std::min(4, nq[s] - op.n + 1));
          std::vector<int> ins;
          for (int q = 0; q < op.n; ++q) {
            op.t[q] = perm[q];
            ins.push_back(perm[q]);
          }
          for (int c = 0; c < nc; ++c) {
            op.ctrl |= 1u << perm[op.n + c];
            ins.push_back(perm[op.n + c]);
          }
          std::sort(ins.begin(), ins.end());
          op.nins = (int)ins.size();
          for (int i = 0; i < op.nins; ++i) op.ins[i] = (int8_t)ins[i];
        } else if (op.kind == 1) {
          op.n = 1 + (int)(rng() % 3);
          for (int q = 0; q < op.n; ++q) op.t[q] = perm[q];
        } else {
          const int w = 1 + (int)(rng() % (it % 5 == 0 ? nq[s] : 6));   // sometimes wider than a tile
          for (int q = 0; q < w; ++q) {
            const int pauli = 1 + (int)(rng() % 3);
            if (pauli != 3) op.xy |= 1u << perm[q];
            if (pauli != 1) op.yz |= 1u << perm[q];
          }
          op.h = op.xy ? 31 - __builtin_clz(op.xy) : 0;
        }
        ops.push_back(op);
      }
      states[s].nops = n_ops;
    }
    std::vector<qsk::BatchSeg> segs;
    std::vector<qsk::BatchXlat> xlat;
    qsbatch::build_segments(L, nq, states, ops, segs, xlat);
    for (int s = 0; s < S; ++s) {
      const qsk::BatchState& st = states[s];
      if (nq[s] <= L) {
        CHECK(st.nsegs == 0, "state fits but has segments");
        continue;
      }
      // the segments cover the state's operations in order, without gaps
      int next = st.first_op;
      for (int g = st.first_seg; g < st.first_seg + st.nsegs; ++g) {
        const qsk::BatchSeg& seg = segs[g];
        CHECK(seg.first_op == next && seg.nops >= 1, "segment order");
        next += seg.nops;
        if (seg.L == 0) {
          CHECK(seg.nops == 1, "a global segment holds one operation");
          CHECK(qsbatch::popc32(31u | qsbatch::pairing_mask(ops[seg.first_op])) > L, "global only when wider");
          continue;
        }
        CHECK(seg.L == L, "tile size");
        uint32_t Q = 0;
        for (int b = 0; b < L; ++b) {
          CHECK(seg.q[b] >= 0 && seg.q[b] < nq[s], "tile qubit range");
          if (b) CHECK(seg.q[b] > seg.q[b - 1], "tile qubits ascending");
          Q |= 1u << seg.q[b];
        }
        CHECK((Q & 31u) == 31u, "the five lowest qubits are tile qubits");
        for (int k = seg.first_op; k < seg.first_op + seg.nops; ++k) {
          const qsk::BatchOp& op = ops[k];
          const qsk::BatchXlat& x = xlat[k];
          CHECK((qsbatch::pairing_mask(op) & ~Q) == 0u, "pairing qubits inside the tile");
          if (op.kind == 0) {
            std::vector<int> want;
            for (int q = 0; q < op.n; ++q) {
              CHECK(x.lt[q] == qsbatch::local_pos(Q, op.t[q]), "dense target position");
              want.push_back(x.lt[q]);
            }
            CHECK((x.fctrl & Q) == 0u && (x.fctrl | (op.ctrl & Q)) == op.ctrl, "controls split");
            uint32_t lc = 0;
            for (int c = 0; c < 32; ++c)
              if (((op.ctrl & Q) >> c) & 1u) {
                lc |= 1u << qsbatch::local_pos(Q, c);
                want.push_back(qsbatch::local_pos(Q, c));
              }
            CHECK(x.lctrl == lc, "local controls");
            std::sort(want.begin(), want.end());
            CHECK(x.nlins == (int)want.size(), "insertion count");
            for (int i = 0; i < x.nlins && i < (int)want.size(); ++i) CHECK(x.lins[i] == want[i], "insertion positions");
          } else if (op.kind == 1) {
            for (int q = 0; q < op.n; ++q) CHECK(x.lt[q] == qsbatch::local_pos(Q, op.t[q]), "diagonal target position");
          } else {
            CHECK(qsbatch::popc32(x.lxy) == qsbatch::popc32(op.xy), "flip mask size");
            CHECK((x.fyz & Q) == 0u && qsbatch::popc32(x.lyz) + qsbatch::popc32(x.fyz) == qsbatch::popc32(op.yz),
                  "phase mask split");
            if (op.xy) CHECK(x.lh == qsbatch::local_pos(Q, op.h), "highest flip bit");
          }
        }
      }
      CHECK(next == st.first_op + st.nops, "segments cover the program");
    }
  }
  std::printf("plan ok (%d failures)\n", failures);
}

int main() {
  std::string line;
  while (std::getline(std::cin, line)) {
    std::istringstream in(line);
    std::string cmd;
    in >> cmd;
    if (cmd == "plan") {
      check_plan();
    } else if (cmd == "c1") {
      double f[4];
      in >> f[0] >> f[1] >> f[2] >> f[3];
      print(qsbatch::channel1_superop(f[0], f[1], f[2], f[3]));
    } else if (cmd == "damp") {
      double p;
      in >> p;
      print(qsbatch::damping_superop(p));
    } else if (cmd == "c2") {
      int depol;
      double p;
      in >> depol >> p;
      print(qsbatch::channel2_superop(depol != 0, p));
    } else if (cmd == "kraus") {
      int n, m;
      in >> n >> m;
      std::vector<double> k((size_t)2 * m << (2 * n));
      for (double& v : k) in >> v;
      print(qsbatch::kraus_superop(n, k.data(), m));
    }
  }
  return failures ? 1 : 0;
}
