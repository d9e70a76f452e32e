// Circuits with gate fusion (C ABI, include/qs.h).
//
// A circuit is a list of unitary operations: many-control many-target dense
// gates, diagonals and Pauli gadgets.  A plan cuts it into blocks of
// consecutive gates that together touch at most max_block_qubits qubits.  A
// block of two or more gates is composed on the device into one dense matrix
// in FP64 (k_block_compose) and applied as a single dense gate, on the tensor
// cores for complex64 states (3..5 qubits) and in double-float arithmetic for
// complex128; a block of one gate is applied by that gate's own kernel.  The
// plan changes only how the work is grouped, not the operation applied: the
// result equals the gate-by-gate result up to rounding.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "qs.h"
#include "qs_handle.h"
#include "qs_alloc.h"
#include "qs_internal.h"

namespace {

struct CGate {
  int kind = 0;                 // 0 dense (controls, targets, matrix), 1 diagonal, 2 Pauli gadget
  std::vector<int> ctrls, targs, paulis;
  std::vector<double> data;     // matrix or diagonal, complex128 (re, im)
  double theta = 0.0;
  uint64_t qmask = 0;           // every qubit the gate touches
};

struct CBlock {
  int first = 0, last = 0;      // gates [first, last)
  std::vector<int> qubits;      // block bit q <-> qubit qubits[q]
  bool fused = false;
  size_t mat_off = 0;           // offset (doubles) of the composed matrix
};

int popc64(uint64_t x) { return __builtin_popcountll(x); }

}  // namespace

struct qs_circuit {
  int nq = 0;
  std::vector<CGate> gates;
  std::vector<CBlock> blocks;
  bool planned = false;
  double* d_mats = nullptr;
  size_t mats_bytes = 0;
  // lazy relabelling (qs_circuit_plan_relabel): physical SWAPs before each
  // block, and the SWAPs that restore the identity layout after the last
  bool relabel = false;
  std::vector<std::vector<std::pair<int, int>>> swaps_before;
  std::vector<std::pair<int, int>> swaps_after;
};

namespace {

void free_device(qs_circuit* c) {
  if (c->d_mats) cudaFree(c->d_mats);
  c->d_mats = nullptr;
  c->mats_bytes = 0;
}

qs_status add_gate(qs_circuit* c, CGate&& g) {
  for (int q : g.targs) g.qmask |= 1ull << q;
  for (int q : g.ctrls) g.qmask |= 1ull << q;
  c->gates.push_back(std::move(g));
  c->planned = false;
  c->relabel = false;
  return QS_OK;
}

// Build the compose instructions of every fused block, compose on the device
// (default stream of the current device, synchronously) and keep the
// matrices.
qs_status compose(qs_circuit* c) {
  free_device(c);
  std::vector<qsk::ComposeBlock> cb;
  std::vector<qsk::ComposeInstr> ins;
  std::vector<double> data;
  size_t out_doubles = 0;
  for (CBlock& b : c->blocks) {
    if (!b.fused) continue;
    const int k = (int)b.qubits.size();
    auto local = [&](int q) { return (int)(std::find(b.qubits.begin(), b.qubits.end(), q) - b.qubits.begin()); };
    qsk::ComposeBlock blk{};
    blk.k = k;
    blk.first = (int)ins.size();
    for (int gi = b.first; gi < b.last; ++gi) {
      const CGate& g = c->gates[gi];
      qsk::ComposeInstr in{};
      in.kind = g.kind;
      if (g.kind == 2) {
        int ny = 0;
        for (size_t q = 0; q < g.targs.size(); ++q) {
          const int p = g.paulis[q], lb = local(g.targs[q]);
          if (p == 1 || p == 2) in.xy |= 1 << lb;
          if (p == 2 || p == 3) in.yz |= 1 << lb;
          if (p == 2) ++ny;
        }
        in.eta = ny & 3;
        const double phi = -0.5 * g.theta;
        in.c = std::cos(phi);
        in.s = std::sin(phi);
      } else {
        in.n = (int)g.targs.size();
        for (int q = 0; q < in.n; ++q) in.tbit[q] = local(g.targs[q]);
        for (int q : g.ctrls) in.ctrl_mask |= 1 << local(q);
        in.data_off = (int)data.size();
        data.insert(data.end(), g.data.begin(), g.data.end());
      }
      ins.push_back(in);
    }
    blk.count = (int)ins.size() - blk.first;
    blk.out_off = (int)out_doubles;
    b.mat_off = out_doubles;
    out_doubles += 2 * (size_t(1) << (2 * k));
    cb.push_back(blk);
  }
  if (cb.empty()) return QS_OK;
  qsk::ComposeBlock* d_cb = nullptr;
  qsk::ComposeInstr* d_ins = nullptr;
  double* d_data = nullptr;
  qs_status st = QS_OK;
  if (qsalloc::device(reinterpret_cast<void**>(&c->d_mats), out_doubles * sizeof(double)) != cudaSuccess ||
      qsalloc::device(reinterpret_cast<void**>(&d_cb), cb.size() * sizeof(qsk::ComposeBlock)) != cudaSuccess ||
      qsalloc::device(reinterpret_cast<void**>(&d_ins), ins.size() * sizeof(qsk::ComposeInstr)) != cudaSuccess ||
      qsalloc::device(reinterpret_cast<void**>(&d_data), std::max<size_t>(1, data.size()) * sizeof(double)) != cudaSuccess) {
    st = QS_ERR_OOM;
  }
  if (st == QS_OK) {
    c->mats_bytes = out_doubles * sizeof(double);
    if (cudaMemcpy(d_cb, cb.data(), cb.size() * sizeof(qsk::ComposeBlock), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_ins, ins.data(), ins.size() * sizeof(qsk::ComposeInstr), cudaMemcpyHostToDevice) != cudaSuccess ||
        (!data.empty() &&
         cudaMemcpy(d_data, data.data(), data.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) ||
        qsk::launch_block_compose(d_cb, (int)cb.size(), d_ins, d_data, c->d_mats, nullptr) != cudaSuccess ||
        cudaStreamSynchronize(nullptr) != cudaSuccess)
      st = QS_ERR_CUDA;
  }
  if (d_cb) cudaFree(d_cb);
  if (d_ins) cudaFree(d_ins);
  if (d_data) cudaFree(d_data);
  if (st != QS_OK) {
    cudaGetLastError();
    free_device(c);
  }
  return st;
}

void close_block(qs_circuit* c, int first, int last, uint64_t mask) {
  CBlock b;
  b.first = first;
  b.last = last;
  for (int q = 0; q < 64; ++q)
    if (mask >> q & 1) b.qubits.push_back(q);
  b.fused = (last - first) >= 2;
  c->blocks.push_back(std::move(b));
}

}  // namespace

// Planner shared with the cost-model planner (qs_costmodel.cpp): cut points
// given as the first gate of every block.
qs_status qs_circuit_set_blocks_internal(qs_circuit* c, const std::vector<int>& starts, int max_block_qubits) {
  c->blocks.clear();
  c->relabel = false;
  c->swaps_before.clear();
  c->swaps_after.clear();
  const int G = (int)c->gates.size();
  for (size_t i = 0; i < starts.size(); ++i) {
    const int first = starts[i], last = i + 1 < starts.size() ? starts[i + 1] : G;
    uint64_t mask = 0;
    for (int g = first; g < last; ++g) mask |= c->gates[g].qmask;
    if (last - first >= 2 && popc64(mask) > max_block_qubits) return QS_ERR_ARG;
    close_block(c, first, last, mask);
  }
  qs_status st = compose(c);
  c->planned = st == QS_OK;
  return st;
}

extern "C" {

qs_status qs_circuit_create(int num_qubits, qs_circuit** out) {
  if (!out || num_qubits < 1 || num_qubits > QS_MAX_STORAGE_QUBITS) return QS_ERR_ARG;
  qs_circuit* c = new (std::nothrow) qs_circuit();
  if (!c) return QS_ERR_OOM;
  c->nq = num_qubits;
  *out = c;
  return QS_OK;
}

qs_status qs_circuit_destroy(qs_circuit* c) {
  if (!c) return QS_ERR_ARG;
  free_device(c);
  delete c;
  return QS_OK;
}

qs_status qs_circuit_add_unitary(qs_circuit* c, const int* ctrls, int nctrl, const int* targs, int ntarg,
                                 const double* mat) {
  if (!c || !mat || ntarg < 1) return QS_ERR_ARG;
  if (ntarg > QS_MAX_DENSE_TARGETS) return QS_ERR_TOO_MANY_TARGETS;
  qs_status st = qsapi::check_qubits(c->nq, targs, ntarg, ctrls, nctrl);
  if (st != QS_OK) return st;
  CGate g;
  g.kind = 0;
  g.ctrls.assign(ctrls, ctrls + nctrl);
  g.targs.assign(targs, targs + ntarg);
  g.data.assign(mat, mat + 2 * (size_t(1) << (2 * ntarg)));
  return add_gate(c, std::move(g));
}

qs_status qs_circuit_add_diagonal(qs_circuit* c, const int* targs, int ntarg, const double* diag) {
  if (!c || !diag || ntarg < 1) return QS_ERR_ARG;
  if (ntarg > QS_MAX_DENSE_TARGETS) return QS_ERR_TOO_MANY_TARGETS;
  qs_status st = qsapi::check_qubits(c->nq, targs, ntarg, nullptr, 0);
  if (st != QS_OK) return st;
  CGate g;
  g.kind = 1;
  g.targs.assign(targs, targs + ntarg);
  g.data.assign(diag, diag + 2 * (size_t(1) << ntarg));
  return add_gate(c, std::move(g));
}

qs_status qs_circuit_add_pauli_gadget(qs_circuit* c, const int* targs, const int* paulis, int n, double theta) {
  if (!c || n < 0 || (n > 0 && (!targs || !paulis))) return QS_ERR_ARG;
  qs_status st = qsapi::check_qubits(c->nq, targs, n, nullptr, 0);
  if (st != QS_OK) return st;
  for (int q = 0; q < n; ++q)
    if (paulis[q] < 0 || paulis[q] > 3) return QS_ERR_ARG;
  CGate g;
  g.kind = 2;
  g.targs.assign(targs, targs + n);
  g.paulis.assign(paulis, paulis + n);
  g.theta = theta;
  return add_gate(c, std::move(g));
}

qs_status qs_circuit_plan(qs_circuit* c, int kind, int max_block_qubits) {
  if (!c) return QS_ERR_ARG;
  if (max_block_qubits < 1 || max_block_qubits > QS_MAX_DENSE_TARGETS) return QS_ERR_ARG;
  std::vector<int> starts;
  const int G = (int)c->gates.size();
  if (kind == QS_PLAN_NONE) {
    for (int g = 0; g < G; ++g) starts.push_back(g);
  } else if (kind == QS_PLAN_GREEDY) {
    // extend the current block while the union of touched qubits fits
    uint64_t mask = 0;
    for (int g = 0; g < G; ++g) {
      const uint64_t m = c->gates[g].qmask;
      if (starts.empty() || popc64(mask | m) > max_block_qubits) {
        starts.push_back(g);
        mask = m;
      } else {
        mask |= m;
      }
    }
  } else {
    return QS_ERR_ARG;
  }
  return qs_circuit_set_blocks_internal(c, starts, max_block_qubits);
}

qs_status qs_circuit_plan_cost(qs_circuit* c, qs_costmodel* model, const qs_state* s, int max_block_qubits,
                               int window) {
  if (!c || !model || !s || s->nq != c->nq) return QS_ERR_ARG;
  if (max_block_qubits < 1 || max_block_qubits > QS_MAX_DENSE_TARGETS || window < 2) return QS_ERR_ARG;
  const int G = (int)c->gates.size();
  const int F = QS_COST_FEATURES;
  // Feature rows: every gate run unfused, then every candidate block [i, j).
  std::vector<float> X;
  auto push = [&](int kind, int width, uint64_t mask, int nctrl, int weight) {
    X.resize(X.size() + F);
    return qs_costmodel_encode(kind, width, mask, nctrl, weight, s, X.data() + X.size() - F);
  };
  for (const CGate& g : c->gates) {
    qs_status st;
    if (g.kind == 0)
      st = push(g.targs.size() == 1 ? QS_COST_GATE1 : QS_COST_DENSE, (int)g.targs.size(), g.qmask,
                (int)g.ctrls.size(), 0);
    else if (g.kind == 1)
      st = push(QS_COST_DIAGONAL, (int)g.targs.size(), g.qmask, 0, 0);
    else {
      bool flips = false;
      for (int p : g.paulis) flips |= (p == 1 || p == 2);
      st = push(flips ? QS_COST_GADGET : QS_COST_PHASE, 0, g.qmask, 0, (int)g.targs.size());
    }
    if (st != QS_OK) return st;
  }
  struct Cand {
    int i, j;
  };
  std::vector<Cand> cand;
  for (int i = 0; i < G; ++i) {
    uint64_t mask = c->gates[i].qmask;
    for (int j = i + 2; j <= G && j - i <= window; ++j) {
      mask |= c->gates[j - 1].qmask;
      if (popc64(mask) > max_block_qubits) break;
      cand.push_back({i, j});
      const qs_status st = push(QS_COST_FUSED_DENSE, popc64(mask), mask, 0, 0);
      if (st != QS_OK) return st;
    }
  }
  const int rows = (int)(X.size() / F);
  std::vector<float> pred(rows);
  qs_status st = qs_costmodel_predict(model, X.data(), rows, pred.data());
  if (st != QS_OK) return st;
  // best[j]: least predicted time (ms) of gates [0, j)
  std::vector<double> best(G + 1, 1e300);
  std::vector<int> from(G + 1, -1);
  best[0] = 0.0;
  std::vector<std::vector<std::pair<int, double>>> ending(G + 1);
  for (size_t k = 0; k < cand.size(); ++k) ending[cand[k].j].push_back({cand[k].i, std::exp((double)pred[G + k])});
  for (int j = 1; j <= G; ++j) {
    best[j] = best[j - 1] + std::exp((double)pred[j - 1]);
    from[j] = j - 1;
    for (const auto& e : ending[j])
      if (best[e.first] + e.second < best[j]) {
        best[j] = best[e.first] + e.second;
        from[j] = e.first;
      }
  }
  std::vector<int> starts;
  for (int j = G; j > 0; j = from[j]) starts.push_back(from[j]);
  std::reverse(starts.begin(), starts.end());
  return qs_circuit_set_blocks_internal(c, starts, max_block_qubits);
}

qs_status qs_circuit_plan_relabel(qs_circuit* c, qs_costmodel* model, const qs_state* s, int low_qubits,
                                  double swap_passes) {
  if (!c || !model || !s || s->nq != c->nq || low_qubits < 0 || low_qubits >= c->nq) return QS_ERR_ARG;
  if (!c->planned) return QS_ERR_ARG;
  const int B = (int)c->blocks.size(), nq = c->nq;
  c->relabel = false;
  c->swaps_before.assign((size_t)B, {});
  c->swaps_after.clear();
  if (low_qubits == 0 || s->is_density) return QS_OK;
  // per block: its qubits, and its launch if it runs on the tensor cores
  // (the only kernels whose speed depends on where the qubits lie)
  std::vector<uint64_t> bmask((size_t)B, 0);
  std::vector<int> tc((size_t)B, 0), kind((size_t)B, 0), width((size_t)B, 0), nctrl((size_t)B, 0);
  for (int b = 0; b < B; ++b) {
    const CBlock& bl = c->blocks[(size_t)b];
    for (int q : bl.qubits) bmask[(size_t)b] |= 1ull << q;
    if (bl.fused) {
      kind[(size_t)b] = QS_COST_FUSED_DENSE;
      width[(size_t)b] = popc64(bmask[(size_t)b]);
      tc[(size_t)b] = width[(size_t)b] >= 2;
    } else {
      const CGate& g = c->gates[(size_t)bl.first];
      if (g.kind == 0 && g.targs.size() >= 2) {
        kind[(size_t)b] = QS_COST_DENSE;
        width[(size_t)b] = (int)g.targs.size();
        nctrl[(size_t)b] = (int)g.ctrls.size();
        tc[(size_t)b] = 1;
      }
    }
  }
  std::vector<float> row(QS_COST_FEATURES);
  auto predict_ms = [&](int k, int w, uint64_t mask, int nc, double* out) {
    qs_status st = qs_costmodel_encode(k, w, mask, nc, 0, s, row.data());
    float y = 0.0f;
    if (st == QS_OK) st = qs_costmodel_predict(model, row.data(), 1, &y);
    *out = std::exp((double)y);
    return st;
  };
  // the price of a SWAP pass, in predicted one-target passes
  double swap_ms = 0.0;
  qs_status st = predict_ms(QS_COST_GATE1, 1, 1ull << (nq - 1), 0, &swap_ms);
  if (st != QS_OK) return st;
  swap_ms *= swap_passes;
  std::vector<int> perm((size_t)nq), inv((size_t)nq);
  for (int q = 0; q < nq; ++q) perm[(size_t)q] = inv[(size_t)q] = q;
  auto physical = [&](uint64_t m) {
    uint64_t r = 0;
    for (int q = 0; q < nq; ++q)
      if (m >> q & 1) r |= 1ull << perm[(size_t)q];
    return r;
  };
  auto do_swap = [&](int p1, int p2, std::vector<std::pair<int, int>>& into) {
    into.push_back({p1, p2});
    const int q1 = inv[(size_t)p1], q2 = inv[(size_t)p2];
    perm[(size_t)q1] = p2;
    perm[(size_t)q2] = p1;
    inv[(size_t)p1] = q2;
    inv[(size_t)p2] = q1;
  };
  const uint64_t lowmask = (1ull << low_qubits) - 1;
  int nswaps = 0;
  for (int b = 0; b < B; ++b) {
    if (!tc[(size_t)b]) continue;
    for (;;) {
      const uint64_t pm = physical(bmask[(size_t)b]);
      const uint64_t bad = pm & lowmask;
      if (!bad) break;
      const int plow = __builtin_ctzll(bad);
      // the high position whose qubit the tensor-core blocks need last (or never)
      int best_p = -1, best_next = -1;
      for (int p = low_qubits; p < nq; ++p) {
        const int q = inv[(size_t)p];
        if (bmask[(size_t)b] >> q & 1) continue;
        int next = B + 1;
        for (int b2 = b + 1; b2 < B; ++b2)
          if (tc[(size_t)b2] && (bmask[(size_t)b2] >> q & 1)) {
            next = b2;
            break;
          }
        if (next >= best_next) {
          best_next = next;
          best_p = p;
        }
      }
      if (best_p < 0) break;
      double t_now = 0.0, t_after = 0.0;
      st = predict_ms(kind[(size_t)b], width[(size_t)b], pm, nctrl[(size_t)b], &t_now);
      if (st == QS_OK)
        st = predict_ms(kind[(size_t)b], width[(size_t)b], (pm & ~(1ull << plow)) | (1ull << best_p),
                        nctrl[(size_t)b], &t_after);
      if (st != QS_OK) return st;
      if (t_now - t_after <= swap_ms) break;
      do_swap(plow, best_p, c->swaps_before[(size_t)b]);
      ++nswaps;
    }
  }
  // back to the identity layout: physical p receives logical p
  for (int p = 0; p < nq; ++p)
    if (inv[(size_t)p] != p) {
      do_swap(p, perm[(size_t)p], c->swaps_after);
      ++nswaps;
    }
  c->relabel = nswaps > 0;
  return QS_OK;
}

qs_status qs_circuit_get_relabel(const qs_circuit* c, int* num_swaps) {
  if (!c || !num_swaps) return QS_ERR_ARG;
  int n = (int)c->swaps_after.size();
  for (const auto& v : c->swaps_before) n += (int)v.size();
  *num_swaps = c->relabel ? n : 0;
  return QS_OK;
}

qs_status qs_circuit_get_plan(const qs_circuit* c, int* num_gates, int* num_blocks, int* num_fused) {
  if (!c) return QS_ERR_ARG;
  int fused = 0;
  for (const CBlock& b : c->blocks) fused += b.fused ? 1 : 0;
  if (num_gates) *num_gates = (int)c->gates.size();
  if (num_blocks) *num_blocks = (int)c->blocks.size();
  if (num_fused) *num_fused = fused;
  return QS_OK;
}

qs_status qs_circuit_apply(qs_circuit* c, qs_state* s) {
  if (!c || !s) return QS_ERR_ARG;
  if (s->nq != c->nq) return QS_ERR_ARG;
  if (!c->planned) {
    const qs_status st = qs_circuit_plan(c, QS_PLAN_NONE, 1);
    if (st != QS_OK) return st;
  }
  // lazy relabelling: logical qubit q lives at physical position perm[q]
  const bool rl = c->relabel && !s->is_density && c->swaps_before.size() == c->blocks.size();
  std::vector<int> perm((size_t)c->nq), inv((size_t)c->nq);
  for (int q = 0; q < c->nq; ++q) perm[(size_t)q] = inv[(size_t)q] = q;
  auto swap_phys = [&](int p1, int p2) {
    const qs_status st = qs_apply_swap(s, p1, p2);
    const int q1 = inv[(size_t)p1], q2 = inv[(size_t)p2];
    perm[(size_t)q1] = p2;
    perm[(size_t)q2] = p1;
    inv[(size_t)p1] = q2;
    inv[(size_t)p2] = q1;
    return st;
  };
  auto mapped = [&](const std::vector<int>& v) {
    std::vector<int> r(v);
    if (rl)
      for (int& q : r) q = perm[(size_t)q];
    return r;
  };
  for (size_t bi = 0; bi < c->blocks.size(); ++bi) {
    const CBlock& b = c->blocks[bi];
    qs_status st = QS_OK;
    if (rl)
      for (const auto& sw : c->swaps_before[bi]) {
        st = swap_phys(sw.first, sw.second);
        if (st != QS_OK) return st;
      }
    if (b.fused) {
      const double* m = c->d_mats + b.mat_off;
      std::vector<int> t = mapped(b.qubits);
      st = qsapi::gate_pass(s, {}, t, nullptr, m, 0, true);
      if (st == QS_OK && s->is_density) {
        for (int& q : t) q += s->nq;
        st = qsapi::gate_pass(s, {}, t, nullptr, m, 1, true);
      }
    } else {
      const CGate& g = c->gates[b.first];
      const std::vector<int> ct = mapped(g.ctrls), tg = mapped(g.targs);
      if (g.kind == 0)
        st = qs_apply_ctrl_multi_target(s, ct.data(), (int)ct.size(), tg.data(), (int)tg.size(), g.data.data());
      else if (g.kind == 1)
        st = qs_apply_diagonal(s, tg.data(), (int)tg.size(), g.data.data());
      else
        st = qs_apply_pauli_gadget(s, tg.data(), g.paulis.data(), (int)tg.size(), g.theta);
    }
    if (st != QS_OK) return st;
  }
  if (rl)
    for (const auto& sw : c->swaps_after) {
      const qs_status st = swap_phys(sw.first, sw.second);
      if (st != QS_OK) return st;
    }
  return QS_OK;
}

}  // extern "C"
