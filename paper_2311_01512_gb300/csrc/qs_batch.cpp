// Batched engine (C ABI, include/qs.h): many independent statevectors with
// their own circuits, run by one persistent kernel launch (qs_batch_kernels.cu)
// that is captured once in a CUDA graph and replayed.
//
// Scheduling: states are ordered by estimated work (amplitudes x operations),
// largest first, and CTAs take them from a shared counter, so the long states
// start early and the short ones fill the gaps (longest-processing-time
// order).  The launch shape (threads per CTA, CTAs per SM, and with it the
// largest state kept in shared memory) is chosen by timing every candidate on
// the batch itself.
//
// States larger than shared memory are cut into segments (cache blocking):
// consecutive operations are grouped while the qubits they pair (dense
// targets, gadget X/Y qubits) together with the five lowest qubits fit in a
// tile of L qubits; the kernel then moves each tile through shared memory once
// per segment instead of moving the state once per operation.
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
#include "qs_batch_plan.h"

struct qs_batch {
  qs_prec prec = QS_C64;
  cudaStream_t stream = nullptr;
  std::vector<int> nq;          // storage qubits (2N for a density matrix)
  std::vector<int> nlog;        // N: the qubits operations name
  std::vector<int> dens;        // density matrix (Choi vector) or statevector
  std::vector<size_t> offset;  // amplitudes
  size_t pool_amps = 0;
  void* pool = nullptr;
  std::vector<std::vector<qsk::BatchOp>> progs;
  std::vector<std::vector<double>> consts;   // per state; BatchOp::coff indexes it until compile
  qsk::BatchState* d_states = nullptr;
  qsk::BatchSeg* d_segs = nullptr;
  qsk::BatchXlat* d_xlat = nullptr;
  int* d_order = nullptr;
  qsk::BatchOp* d_ops = nullptr;
  double* d_consts = nullptr;
  int* d_counter = nullptr;
  long num_segs = 0;
  int wide = 0;                 // some operation is dense on 3 or 4 targets
  int threads = 256, ctas = 0, smem_qubits = -1;
  cudaStream_t capture_stream = nullptr;  // own stream for recording (the caller's may be the legacy stream)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool compiled = false;
  long total_ops = 0;
  float best_ms = 0.f;
};

namespace {

void free_device(qs_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (void* p : {(void*)b->d_states, (void*)b->d_segs, (void*)b->d_xlat, (void*)b->d_order, (void*)b->d_ops,
                  (void*)b->d_consts, (void*)b->d_counter})
    if (p) cudaFree(p);
  b->d_consts = nullptr;
  b->exec = nullptr;
  b->graph = nullptr;
  b->d_states = nullptr;
  b->d_segs = nullptr;
  b->d_xlat = nullptr;
  b->d_order = nullptr;
  b->d_ops = nullptr;
  b->d_counter = nullptr;
  b->compiled = false;
}

qs_status check_state(const qs_batch* b, int s) {
  if (!b || s < 0 || s >= (int)b->nq.size()) return QS_ERR_ARG;
  return QS_OK;
}

// one operation on storage qubits, with its nc constants
qs_status add(qs_batch* b, int s, qsk::BatchOp op, const double* c, size_t nc) {
  op.coff = b->consts[s].size();
  b->consts[s].insert(b->consts[s].end(), c, c + nc);
  b->progs[s].push_back(op);
  b->compiled = false;
  return QS_OK;
}

// dense operation on storage targets t (matrix bit q on t[q]) with storage controls c
qs_status add_dense(qs_batch* b, int s, const std::vector<int>& c, const std::vector<int>& t, const double* mat) {
  qsk::BatchOp op{};
  op.kind = 0;
  op.n = (int)t.size();
  std::vector<int> ins(t);
  for (int q = 0; q < op.n; ++q) op.t[q] = t[q];
  for (int q : c) {
    op.ctrl |= 1u << q;
    ins.push_back(q);
  }
  if (ins.size() > 7) return QS_ERR_TOO_MANY_TARGETS;
  std::sort(ins.begin(), ins.end());
  op.nins = (int)ins.size();
  for (int i = 0; i < op.nins; ++i) op.ins[i] = (int8_t)ins[i];
  return add(b, s, op, mat, (size_t)2 << (2 * op.n));
}

// Superoperator of a channel on the Choi vector as a dense operation on
// (t, t + N) (one qubit) or (t1, t2, t1 + N, t2 + N) (two qubits): member m
// has bit q of m on the q-th of those positions; S (real, row-major, d x d)
// gives new beta_m = sum_k S[m][k] beta_k.
qs_status add_superop(qs_batch* b, int s, const std::vector<int>& targs, const std::vector<double>& S) {
  const int n = (int)targs.size(), d = 1 << (2 * n);
  std::vector<int> t(targs);
  for (int q = 0; q < n; ++q) t.push_back(targs[q] + b->nlog[s]);
  std::vector<double> m((size_t)2 * d * d, 0.0);
  for (int i = 0; i < d * d; ++i) m[2 * i] = S[i];
  return add_dense(b, s, {}, t, m.data());
}

qs_status check_density(const qs_batch* b, int s) {
  if (check_state(b, s) != QS_OK) return QS_ERR_ARG;
  return b->dens[s] ? QS_OK : QS_ERR_NOT_DENSMATR;
}

qs_status check_prob(double p) { return (p >= 0.0 && p <= 1.0) ? QS_OK : QS_ERR_ARG; }

// One-qubit channels in the paper's Choi-vector form: members 00 and 11 (bits
// t, t + N) mix as f0 self + f1 other; 01 and 10 as f2 self + f3 other.
qs_status add_channel1(qs_batch* b, int s, int t, double f0, double f1, double f2, double f3) {
  if (check_density(b, s) != QS_OK) return check_density(b, s);
  qs_status st = qsapi::check_qubits(b->nlog[s], &t, 1, nullptr, 0);
  if (st != QS_OK) return st;
  return add_superop(b, s, {t}, qsbatch::channel1_superop(f0, f1, f2, f3));
}

int smem_qubits_for(qs_prec prec, int ctas_per_sm) {
  const size_t per_cta = std::min<size_t>(200 * 1024 / ctas_per_sm, 200 * 1024);
  const size_t amp = prec == QS_C128 ? 16 : 8;
  int q = 0;
  while (((size_t)1 << (q + 1)) * amp <= per_cta) ++q;
  return q;
}

// ---- segment plans (for one tile size L) ------------------------------------
struct Plan {
  int L = -1;
  std::vector<qsk::BatchState> states;
  std::vector<qsk::BatchSeg> segs;
  std::vector<qsk::BatchXlat> xlat;   // parallel to the operations
  qsk::BatchState* d_states = nullptr;
  qsk::BatchSeg* d_segs = nullptr;
  qsk::BatchXlat* d_xlat = nullptr;
  void release() {
    for (void* p : {(void*)d_states, (void*)d_segs, (void*)d_xlat})
      if (p) cudaFree(p);
    d_states = nullptr;
    d_segs = nullptr;
    d_xlat = nullptr;
  }
};

// Segments of every state larger than 2^L amplitudes (qs_batch_plan.h).
void build_plan(Plan& P, int L, const std::vector<int>& nq, const std::vector<qsk::BatchState>& base,
                const std::vector<qsk::BatchOp>& ops) {
  P.L = L;
  P.states = base;
  qsbatch::build_segments(L, nq, P.states, ops, P.segs, P.xlat);
}

bool upload_plan(Plan& P) {
  const size_t S = P.states.size();
  if (qsalloc::device(reinterpret_cast<void**>(&P.d_states), sizeof(qsk::BatchState) * S) != cudaSuccess ||
      qsalloc::device(reinterpret_cast<void**>(&P.d_segs), sizeof(qsk::BatchSeg) * std::max<size_t>(1, P.segs.size())) != cudaSuccess ||
      qsalloc::device(reinterpret_cast<void**>(&P.d_xlat), sizeof(qsk::BatchXlat) * std::max<size_t>(1, P.xlat.size())) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (cudaMemcpy(P.d_states, P.states.data(), sizeof(qsk::BatchState) * S, cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  if (!P.segs.empty() && cudaMemcpy(P.d_segs, P.segs.data(), sizeof(qsk::BatchSeg) * P.segs.size(),
                                    cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  return P.xlat.empty() || cudaMemcpy(P.d_xlat, P.xlat.data(), sizeof(qsk::BatchXlat) * P.xlat.size(),
                                      cudaMemcpyHostToDevice) == cudaSuccess;
}

// Two-qubit channels on the members of (t1, t2, t1 + N, t2 + N): member bits
// 0, 1 are t1, t2 and bits 2, 3 are t1 + N, t2 + N.
qs_status add_channel2(qs_batch* b, int state, int t1, int t2, bool depol, double p) {
  if (check_density(b, state) != QS_OK) return check_density(b, state);
  const int tt[2] = {t1, t2};
  qs_status st = qsapi::check_qubits(b->nlog[state], tt, 2, nullptr, 0);
  if (st != QS_OK) return st;
  return add_superop(b, state, {t1, t2}, qsbatch::channel2_superop(depol, p));
}

}  // namespace

extern "C" {

qs_status qs_batch_create(int num_states, const int* num_qubits, qs_prec prec, void* cuda_stream, qs_batch** out) {
  return qs_batch_create_mixed(num_states, num_qubits, nullptr, prec, cuda_stream, out);
}

qs_status qs_batch_create_mixed(int num_states, const int* num_qubits, const int* is_density, qs_prec prec,
                                void* cuda_stream, qs_batch** out) {
  if (!out || num_states < 1 || !num_qubits || (prec != QS_C64 && prec != QS_C128)) return QS_ERR_ARG;
  *out = nullptr;
  qs_batch* b = new (std::nothrow) qs_batch();
  if (!b) return QS_ERR_OOM;
  b->prec = prec;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->nlog.assign(num_qubits, num_qubits + num_states);
  b->dens.assign(num_states, 0);
  if (is_density)
    for (int s = 0; s < num_states; ++s) b->dens[s] = is_density[s] ? 1 : 0;
  for (int s = 0; s < num_states; ++s) b->nq.push_back(b->dens[s] ? 2 * b->nlog[s] : b->nlog[s]);
  b->progs.resize(num_states);
  b->consts.resize(num_states);
  size_t off = 0;
  for (int s = 0; s < num_states; ++s) {
    const int q = b->nq[s];
    if (b->nlog[s] < 1 || q > 24) {
      delete b;
      return QS_ERR_ARG;
    }
    b->offset.push_back(off);
    off += (size_t)1 << q;
    off = (off + 31) & ~(size_t)31;    // 256-byte aligned starts for complex64 and complex128
  }
  b->pool_amps = off;
  *out = b;
  return QS_OK;
}

qs_status qs_batch_destroy(qs_batch* b) {
  if (!b) return QS_ERR_ARG;
  free_device(b);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  delete b;
  return QS_OK;
}

qs_status qs_batch_pool_amps(const qs_batch* b, size_t* num_amps) {
  if (!b || !num_amps) return QS_ERR_ARG;
  *num_amps = b->pool_amps;
  return QS_OK;
}

qs_status qs_batch_state_offset(const qs_batch* b, int state, size_t* offset_amps) {
  if (check_state(b, state) != QS_OK || !offset_amps) return QS_ERR_ARG;
  *offset_amps = b->offset[state];
  return QS_OK;
}

qs_status qs_batch_bind_pool(qs_batch* b, void* d_pool) {
  if (!b || !d_pool) return QS_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(d_pool) % 256 != 0) return QS_ERR_ALIGN;
  b->pool = d_pool;
  b->compiled = false;
  return QS_OK;
}

qs_status qs_batch_add_unitary(qs_batch* b, int state, const int* ctrls, int nctrl, const int* targs, int ntarg,
                               const double* mat) {
  if (check_state(b, state) != QS_OK || !mat || ntarg < 1) return QS_ERR_ARG;
  if (ntarg > 2 || nctrl > 5) return QS_ERR_TOO_MANY_TARGETS;
  qs_status st = qsapi::check_qubits(b->nlog[state], targs, ntarg, ctrls, nctrl);
  if (st != QS_OK) return st;
  std::vector<int> c(ctrls, ctrls + nctrl), t(targs, targs + ntarg);
  st = add_dense(b, state, c, t, mat);
  if (st != QS_OK || !b->dens[state]) return st;
  // density matrix: U^* on t + N with controls c + N (Sec. "Unitary gates")
  const size_t nm = (size_t)2 << (2 * ntarg);
  std::vector<double> conj(mat, mat + nm);
  for (size_t i = 1; i < nm; i += 2) conj[i] = -conj[i];
  for (int& q : c) q += b->nlog[state];
  for (int& q : t) q += b->nlog[state];
  return add_dense(b, state, c, t, conj.data());
}

qs_status qs_batch_add_diagonal(qs_batch* b, int state, const int* targs, int ntarg, const double* diag) {
  if (check_state(b, state) != QS_OK || !diag || ntarg < 1) return QS_ERR_ARG;
  if (ntarg > 3) return QS_ERR_TOO_MANY_TARGETS;
  qs_status st = qsapi::check_qubits(b->nlog[state], targs, ntarg, nullptr, 0);
  if (st != QS_OK) return st;
  qsk::BatchOp op{};
  op.kind = 1;
  op.n = ntarg;
  for (int q = 0; q < ntarg; ++q) op.t[q] = targs[q];
  const size_t nd = (size_t)2 << ntarg;
  st = add(b, state, op, diag, nd);
  if (st != QS_OK || !b->dens[state]) return st;
  std::vector<double> conj(diag, diag + nd);   // density matrix: conj(d) on t + N
  for (size_t i = 1; i < nd; i += 2) conj[i] = -conj[i];
  for (int q = 0; q < ntarg; ++q) op.t[q] = targs[q] + b->nlog[state];
  return add(b, state, op, conj.data(), nd);
}

qs_status qs_batch_add_pauli_gadget(qs_batch* b, int state, const int* targs, const int* paulis, int n,
                                    double theta) {
  if (check_state(b, state) != QS_OK || n < 0 || (n > 0 && (!targs || !paulis))) return QS_ERR_ARG;
  qs_status st = qsapi::check_qubits(b->nlog[state], targs, n, nullptr, 0);
  if (st != QS_OK) return st;
  for (int q = 0; q < n; ++q)
    if (paulis[q] < 0 || paulis[q] > 3) return QS_ERR_ARG;
  auto one = [&](int shift, double th) {
    qsk::BatchOp op{};
    op.kind = 2;
    int ny = 0;
    for (int q = 0; q < n; ++q) {
      const int t = targs[q] + shift;
      if (paulis[q] == 1 || paulis[q] == 2) op.xy |= 1u << t;
      if (paulis[q] == 2 || paulis[q] == 3) op.yz |= 1u << t;
      if (paulis[q] == 2) ++ny;
    }
    op.eta = ny & 3;
    op.h = op.xy ? 31 - __builtin_clz(op.xy) : 0;
    const double phi = -0.5 * th;
    const double cs[2] = {std::cos(phi), std::sin(phi)};
    return add(b, state, op, cs, 2);
  };
  st = one(0, theta);
  if (st != QS_OK || !b->dens[state]) return st;
  int ny = 0;
  for (int q = 0; q < n; ++q) ny += paulis[q] == 2;
  // U(theta)^* = U((-1)^(#Y + 1) theta) on t + N (Algorithm "specific unitaries on density matrices")
  return one(b->nlog[state], (ny % 2 == 0) ? -theta : theta);
}

qs_status qs_batch_add_kraus(qs_batch* b, int state, const int* targs, int n, const double* kraus, int num_ops) {
  if (check_state(b, state) != QS_OK || !kraus || !targs || num_ops < 1 || n < 1) return QS_ERR_ARG;
  if (!b->dens[state]) return QS_ERR_NOT_DENSMATR;
  if (n > 2) return QS_ERR_TOO_MANY_TARGETS;
  qs_status st = qsapi::check_qubits(b->nlog[state], targs, n, nullptr, 0);
  if (st != QS_OK) return st;
  const std::vector<double> m = qsbatch::kraus_superop(n, kraus, num_ops);
  std::vector<int> t(targs, targs + n);
  for (int q = 0; q < n; ++q) t.push_back(targs[q] + b->nlog[state]);
  return add_dense(b, state, {}, t, m.data());
}

// The channels, in the paper's Choi-vector update rules (Sec. "Dephasing
// channel", "Depolarising channel", "Damping channel"), as superoperators.
qs_status qs_batch_add_dephasing(qs_batch* b, int state, int t, double p) {
  if (check_prob(p) != QS_OK) return QS_ERR_ARG;
  return add_channel1(b, state, t, 1.0, 0.0, 1.0 - 2.0 * p, 0.0);
}

qs_status qs_batch_add_depolarising(qs_batch* b, int state, int t, double p) {
  if (check_prob(p) != QS_OK) return QS_ERR_ARG;
  return add_channel1(b, state, t, 1.0 - 2.0 * p / 3.0, 2.0 * p / 3.0, 1.0 - 4.0 * p / 3.0, 0.0);
}

qs_status qs_batch_add_pauli_channel(qs_batch* b, int state, int t, double px, double py, double pz) {
  if (check_prob(px) != QS_OK || check_prob(py) != QS_OK || check_prob(pz) != QS_OK) return QS_ERR_ARG;
  return add_channel1(b, state, t, 1.0 - px - py, px + py, 1.0 - px - py - 2.0 * pz, px - py);
}

qs_status qs_batch_add_damping(qs_batch* b, int state, int t, double p) {
  if (check_prob(p) != QS_OK) return QS_ERR_ARG;
  if (check_density(b, state) != QS_OK) return check_density(b, state);
  qs_status st = qsapi::check_qubits(b->nlog[state], &t, 1, nullptr, 0);
  if (st != QS_OK) return st;
  return add_superop(b, state, {t}, qsbatch::damping_superop(p));
}

qs_status qs_batch_add_two_qubit_dephasing(qs_batch* b, int state, int t1, int t2, double p) {
  if (check_prob(p) != QS_OK) return QS_ERR_ARG;
  return add_channel2(b, state, t1, t2, false, p);
}

qs_status qs_batch_add_two_qubit_depolarising(qs_batch* b, int state, int t1, int t2, double p) {
  if (check_prob(p) != QS_OK) return QS_ERR_ARG;
  return add_channel2(b, state, t1, t2, true, p);
}

qs_status qs_batch_compile(qs_batch* b, int autotune) {
  if (!b || !b->pool) return QS_ERR_ARG;
  free_device(b);
  const int S = (int)b->nq.size();
  std::vector<qsk::BatchState> states(S);
  std::vector<qsk::BatchOp> ops;
  std::vector<double> consts;
  for (int s = 0; s < S; ++s) {
    states[s].offset = b->offset[s];
    states[s].nq = b->nq[s];
    states[s].first_op = (int)ops.size();
    states[s].nops = (int)b->progs[s].size();
    for (qsk::BatchOp op : b->progs[s]) {
      op.coff += consts.size();
      ops.push_back(op);
    }
    consts.insert(consts.end(), b->consts[s].begin(), b->consts[s].end());
  }
  b->total_ops = (long)ops.size();
  b->wide = 0;
  for (const auto& op : ops)
    if (op.kind == 0 && op.n > 2) b->wide = 1;
  std::vector<int> order(S);
  for (int s = 0; s < S; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return ((double)(1ull << b->nq[x]) * (1 + b->progs[x].size())) >
           ((double)(1ull << b->nq[y]) * (1 + b->progs[y].size()));
  });
  if (qsalloc::device(reinterpret_cast<void**>(&b->d_order), sizeof(int) * S) != cudaSuccess ||
      qsalloc::device(reinterpret_cast<void**>(&b->d_ops), sizeof(qsk::BatchOp) * std::max<size_t>(1, ops.size())) != cudaSuccess ||
      qsalloc::device(reinterpret_cast<void**>(&b->d_consts), sizeof(double) * std::max<size_t>(1, consts.size())) != cudaSuccess ||
      qsalloc::device(reinterpret_cast<void**>(&b->d_counter), sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    free_device(b);
    return QS_ERR_OOM;
  }
  if (cudaMemcpy(b->d_order, order.data(), sizeof(int) * S, cudaMemcpyHostToDevice) != cudaSuccess ||
      (!ops.empty() &&
       cudaMemcpy(b->d_ops, ops.data(), sizeof(qsk::BatchOp) * ops.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
      (!consts.empty() && cudaMemcpy(b->d_consts, consts.data(), sizeof(double) * consts.size(),
                                     cudaMemcpyHostToDevice) != cudaSuccess)) {
    free_device(b);
    return QS_ERR_CUDA;
  }
  // launch-shape candidates: (threads, CTAs per SM); each shared-memory size
  // (tile size) has its own segment plan
  const int sms = qsk::num_sms();
  if (qsk::batch_set_max_smem(200 * 1024) != cudaSuccess) {
    cudaGetLastError();
    return QS_ERR_CUDA;
  }
  std::vector<std::pair<int, int>> cands;
  if (autotune)
    cands = {{128, 4}, {256, 2}, {256, 4}, {512, 1}, {512, 2}};
  else
    cands = {{256, 2}};
  std::vector<Plan> plans;
  plans.reserve(cands.size());       // pointers into it stay valid
  auto plan_for = [&](int L) -> Plan* {
    for (auto& P : plans)
      if (P.L == L) return &P;
    plans.emplace_back();
    build_plan(plans.back(), L, b->nq, states, ops);
    return &plans.back();
  };
  for (const auto& c : cands) {
    Plan* P = plan_for(smem_qubits_for(b->prec, c.second));
    if (!P->d_states && !upload_plan(*P)) {
      for (auto& Q : plans) Q.release();
      free_device(b);
      return QS_ERR_OOM;
    }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int best_plan = -1;
  for (const auto& c : cands) {
    const int sq = smem_qubits_for(b->prec, c.second);
    Plan* P = plan_for(sq);
    if (cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->stream) != cudaSuccess) return QS_ERR_CUDA;
    cudaEventRecord(e0, b->stream);
    if (qsk::launch_batch(b->prec, b->pool, P->d_states, b->d_order, S, b->d_ops, b->d_consts, P->d_segs,
                          P->d_xlat, b->d_counter, c.first, sms * c.second, sq, b->wide, b->stream) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaEventRecord(e1, b->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return QS_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      b->threads = c.first;
      b->ctas = sms * c.second;
      b->smem_qubits = sq;
      best_plan = (int)(P - plans.data());
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int i = 0; i < (int)plans.size(); ++i)
    if (i != best_plan) plans[i].release();
  if (b->ctas == 0 || best_plan < 0) return QS_ERR_CUDA;
  b->d_states = plans[best_plan].d_states;
  b->d_segs = plans[best_plan].d_segs;
  b->d_xlat = plans[best_plan].d_xlat;
  b->num_segs = (long)plans[best_plan].segs.size();
  b->best_ms = best;
  // record on the batch's own stream: reset the work counter, one persistent launch
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return QS_ERR_CUDA;
  if (!b->capture_stream && cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
    return QS_ERR_CUDA;
  if (cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return QS_ERR_CUDA;
  }
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->capture_stream);
  if (e == cudaSuccess)
    e = qsk::launch_batch(b->prec, b->pool, b->d_states, b->d_order, S, b->d_ops, b->d_consts, b->d_segs, b->d_xlat,
                          b->d_counter, b->threads, b->ctas, b->smem_qubits, b->wide, b->capture_stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(b->capture_stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess || !g) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    return QS_ERR_CUDA;
  }
  b->graph = g;
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    return QS_ERR_CUDA;
  }
  b->compiled = true;
  return QS_OK;
}

qs_status qs_batch_run(qs_batch* b) {
  if (!b || !b->compiled) return QS_ERR_ARG;
  return cudaGraphLaunch(b->exec, b->stream) == cudaSuccess ? QS_OK : QS_ERR_CUDA;
}

qs_status qs_batch_info(const qs_batch* b, int* threads, int* ctas, int* smem_qubits, long* total_ops) {
  if (!b) return QS_ERR_ARG;
  if (threads) *threads = b->threads;
  if (ctas) *ctas = b->ctas;
  if (smem_qubits) *smem_qubits = b->smem_qubits;
  if (total_ops) *total_ops = b->total_ops;
  return QS_OK;
}

}  // extern "C"
