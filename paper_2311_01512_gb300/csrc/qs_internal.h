// Internal interface between the C-ABI layer (qs_api.cpp) and the CUDA kernels.
// Host-visible declarations only: parameter structs passed by value to the
// kernels, and one launcher per kernel family.  No torch types anywhere.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "qs.h"

namespace qsk {

constexpr int kMaxQ = QS_MAX_STORAGE_QUBITS;
constexpr int kMaxDense = QS_MAX_DENSE_TARGETS;
constexpr int kTileBits = 10;        // amplitudes staged per tile of the dense kernel: 2^10
constexpr int kReduceBlocks = 1216;  // 152 SMs x 8: fixed grid of the stage-one expectation and trace reductions
constexpr int kNormBlocks = 4864;    // 152 SMs x 32: fixed grid of the norm, a pure stream over the state
constexpr int kPartials = kNormBlocks;  // partial sums a handle holds (the larger grid)
constexpr int kTermChunk = 2048;     // Pauli terms per device upload
constexpr int kCostFeatures = 64;    // cost-model network: input features
constexpr int kCostHidden = 64;      // hidden units per layer (two layers)
constexpr int kCostParams = kCostHidden * kCostFeatures + kCostHidden + kCostHidden * kCostHidden + kCostHidden +
                            kCostHidden + 1;

// One-target gate on pairs (i0, i1 = i0 | 2^t) (Sec. "One-target gate",
// Sec. "Many-control one-target gate").
struct Gate1Params {
  double m[8];           // m00, m01, m10, m11 as (re, im), already conjugated if needed
  uint64_t npairs;       // 2^(Ns - 1 - s)
  uint64_t ctrl_mask;    // control bits, set in every enumerated index
  int t;
  int nins;              // 1 + s
  int8_t ins[kMaxQ];     // sorted target and control positions (zero bits inserted)
};

// The same gate for complex128 with double-float arithmetic: the matrix split
// into float pairs on the host, plus the plain doubles for the share of
// 32-pair chunks (chunk mod f64_mod < f64_count) run in native FP64.
struct Gate1DfParams {
  float mh[8], ml[8];
  double m[8];
  uint64_t npairs;
  uint64_t ctrl_mask;
  int t;
  int nins;
  int f64_mod;
  int f64_count;
  int8_t ins[kMaxQ];
};

// Dense gate on n <= 6 targets staged through shared memory
// (Sec. "Many-target gate").  A tile is the 2^tile_bits amplitudes whose
// indices differ only at the positions P (the targets plus the lowest free
// qubits); the remaining free bits number the tile.
struct DenseParams {
  const double* mat;     // device, 2^n x 2^n complex128 row-major (re, im)
  uint64_t ctrl_mask;
  uint64_t ntiles;
  int n;
  int conj;              // use conj(mat)
  int tile_bits;
  int nhi;
  int8_t tslot[kMaxDense];  // tslot[q]: index within P of target q
  int8_t P[16];             // ascending tile positions
  int8_t hi_ins[kMaxQ];     // sorted (P u controls): zero bits inserted into the tile number
};

// Dense gate on the tensor cores (complex64, 3xTF32): a tile is 128 groups,
// P = the targets plus the 7 lowest free qubits (fewer in small states).
struct TcParams {
  const double* mat;     // device, 2^n x 2^n complex128 row-major (re, im)
  int* err;              // device error word: set to 1 when a bounded wait runs out
  uint64_t ctrl_mask;
  uint64_t ntiles;
  int n;                 // targets of the kernel
  int nmat;              // targets of the stored matrix (< n: identity on targets nmat..n-1)
  int conj;
  int tile_bits;
  int nhi;
  uint32_t tslot_mask;   // bits of P that are targets
  int8_t tslot[kMaxDense];
  int8_t tpos[kMaxDense];
  int8_t P[16];
  int8_t hi_ins[kMaxQ];
};

// Diagonal on n <= 6 targets.
struct DiagParams {
  double d[2 * 64];
  uint64_t namps;
  int n;
  int8_t tpos[kMaxDense];
};

// Pauli gadget / phase gadget (Sec. "Pauli gadget", Sec. "Phase gadget").
struct GadgetParams {
  uint64_t xy;           // qubits with X or Y: the flipped bits
  uint64_t yz;           // qubits with Y or Z: the sign bits
  uint64_t nwork;        // pairs (xy != 0) or amplitudes (xy == 0)
  double c, s;           // cos(phi), sin(phi), phi = -theta/2
  int eta;               // number of Y factors mod 4
  int h;                 // highest bit of xy (pair enumeration)
};

// Gadget parameters for double-float arithmetic: cos(phi), sin(phi) split.
struct GadgetDfParams {
  uint64_t xy, yz, nwork;
  float ch, cl, sh, sl;
  int eta;
  int h;
};

// complex128 kernels in block fixed-point arithmetic (qs_fx.cuh): constants
// prepared on the host as 60-bit fixed-point parts of their row group.
struct FxPart {
  int32_t h, l;          // M = h 2^30 + l, 0 <= l < 2^30
};

// One-target gate: rows r = (out0.re, out0.im, out1.re, out1.im) over the
// columns (a.re, a.im, b.re, b.im) of the pair (a, b); rows 0-1 share the
// exponent em[0] (of m00, m01), rows 2-3 em[1] (of m10, m11).
struct Gate1FxParams {
  FxPart m[4][4];
  int em[2];
  uint64_t npairs;
  uint64_t ctrl_mask;
  int t;
  int nins;
  int8_t ins[kMaxQ];
};

// Two-target gate: rows r = 2 j + (0: re, 1: im) of output amplitude j over
// the columns c = 2 k + (0: re, 1: im) of input amplitude k, j and k = b0 + 2 b1
// with b0 the bit at t0 and b1 the bit at t1; rows 2j and 2j+1 share the
// exponent em[j] (of u_j0 .. u_j3).
struct Gate2FxParams {
  FxPart m[8][8];
  int em[4];
  uint64_t nquads;
  uint64_t ctrl_mask;
  int t0, t1;
  int lo, hi;            // the targets sorted (the no-control index path)
  int nins;
  int8_t ins[kMaxQ];
};

// Diagonal entry d_j: parts of Re, Im and -Im with their shared exponent.
struct DiagFxEntry {
  FxPart re, im, nim;
  int em;
};
struct DiagFxParams {
  DiagFxEntry e[64];
  uint64_t namps;
  int n;
  int8_t tpos[kMaxDense];
};

// Pauli / phase gadget: cos(phi), sin(phi), -sin(phi) with their shared exponent.
struct GadgetFxParams {
  uint64_t xy, yz, nwork;
  FxPart c, s, ns;
  int em;
  int eta;
  int h;
};

// Density-matrix channels acting on groups of 4 (one qubit: bits t, t+N) or 16
// (two qubits: t1, t2, t1+N, t2+N) Choi amplitudes.
enum GroupOp { G_DEPHASE1 = 0, G_DEPHASE2 = 1, G_DEPOL1 = 2, G_DEPOL2 = 3, G_DAMP = 4, G_PAULI1 = 5 };
struct GroupParams {
  uint64_t ngroups;
  int nbits;             // 2 or 4
  int8_t ins[4];         // sorted member positions
  int8_t mpos[4];        // member bit b -> qubit position
  double f[4];           // channel coefficients (see the kernel)
};

// The same channels in block fixed point: coefficient slots with their own
// exponents (which slots an operation uses is stated at its kernel).
struct GroupFxParams {
  uint64_t ngroups;
  int nbits;
  int8_t ins[4];
  int8_t mpos[4];
  FxPart cf[6];
  int em[6];
};

// Partial trace (Sec. "Partial trace").
struct PtraceParams {
  uint64_t nout;         // 2^(2(N - n))
  int n;
  int nins;              // 2n
  int8_t ins[kMaxQ];     // sorted t u (t + N)
  uint64_t pair_mask[kMaxQ / 2 + 1];  // (1 << t[q]) | (1 << (t[q] + N))
};

// One Pauli term of an expectation value.
struct PauliTerm {
  uint64_t xy;
  uint64_t yz;
  double h;
  int eta;               // number of Y factors mod 4
  int pad;
};

// Order in which the statevector expectation visits its tiles of
// 2^kExpecTileBits amplitudes.  The tile-index parts of all flip masks
// (xy >> kExpecTileBits) span a subspace with a reduced basis basis[0..r):
// basis[j] has its highest bit at piv[j] (ascending) and no other pivot bit.
// Virtual tile v = c 2^r + e visits the tile whose pivot bits are e and whose
// other bits are those of c XOR the basis combination e selects: each coset
// of the span is visited in one run of consecutive v, and every partner tile
// (tile xor xy >> kExpecTileBits) lies in the same coset, so it is read while
// the coset is in L2 (when the span is small enough to fit).
constexpr int kExpecTileBits = 10;
struct TileOrder {
  int r;
  int8_t piv[32];
  uint32_t basis[32];
};

inline TileOrder make_tile_order(const PauliTerm* terms, int n) {
  TileOrder o{};
  uint32_t b[32];
  int r = 0;
  for (int k = 0; k < n; ++k) {
    uint32_t v = (uint32_t)(terms[k].xy >> kExpecTileBits);
    for (int j = 0; j < r; ++j)
      if ((v >> (31 - __builtin_clz(b[j]))) & 1u) v ^= b[j];
    if (!v) continue;
    const int p = 31 - __builtin_clz(v);
    for (int j = 0; j < r; ++j)
      if ((b[j] >> p) & 1u) b[j] ^= v;
    b[r++] = v;
  }
  // ascending pivots
  for (int i = 1; i < r; ++i)
    for (int j = i; j > 0 && b[j - 1] > b[j]; --j) {
      const uint32_t t = b[j];
      b[j] = b[j - 1];
      b[j - 1] = t;
    }
  o.r = r;
  for (int j = 0; j < r; ++j) {
    o.basis[j] = b[j];
    o.piv[j] = (int8_t)(31 - __builtin_clz(b[j]));
  }
  return o;
}

// Tile visited at virtual position v: zero bits inserted at the pivots into
// c = v >> r, then the basis vectors selected by the low r bits of v.  So the
// 2^r positions c 2^r .. (c + 1) 2^r - 1 are one coset of the span of the
// basis, the tiles that a term's flip mask pairs with each other.  Host and
// device (the host build is checked on the CPU).
#if defined(__CUDACC__)
__host__ __device__
#endif
inline uint64_t ordered_tile(uint64_t v, const TileOrder& o) {
  const int r = o.r;
  uint64_t t = v >> r;
  for (int j = 0; j < r; ++j) {
    const int p = o.piv[j];
    t = ((t >> p) << (p + 1)) | (t & ((1ull << p) - 1));
  }
  for (int j = 0; j < r; ++j)
    if ((v >> j) & 1) t ^= o.basis[j];
  return t;
}

// Block composition (qs_fuse.cu): one gate of a block, on block-local bits.
struct ComposeInstr {
  int kind;              // 0 dense with controls, 1 diagonal, 2 Pauli gadget
  int n;                 // targets (dense, diagonal)
  int ctrl_mask;         // block-local control bits
  int tbit[kMaxDense];   // block-local bit of target q
  int data_off;          // offset (doubles) of the matrix or diagonal
  int xy, yz, eta;       // gadget: block-local masks, number of Y mod 4
  double c, s;           // gadget: cos(phi), sin(phi), phi = -theta/2
};
struct ComposeBlock {
  int k;                 // block qubits
  int first, count;      // its instructions
  int out_off;           // offset (doubles) of its 2^k x 2^k output matrix
};

// Batched engine (qs_batch_kernels.cu): one operation of a state's program
// and one state (at most 24 qubits: 32-bit indices).
struct BatchOp {
  int kind;              // 0 dense on 1..4 targets with controls, 1 diagonal (<= 3 targets), 2 Pauli gadget
  int n;
  int t[4];
  uint32_t ctrl;         // control mask
  uint32_t xy, yz;       // gadget masks
  int eta, h;            // gadget: number of Y mod 4, highest bit of xy
  int nins;              // dense: sorted target and control positions (at most 7)
  int8_t ins[8];
  uint64_t coff;         // constants in the batch's pool of doubles: dense 2^n x 2^n row-major (re, im),
                         // diagonal 2^n entries, gadget cos(phi), sin(phi)
};
struct BatchState {
  uint64_t offset;       // first amplitude in the pool
  int nq;
  int first_op;
  int nops;
  int first_seg;         // states larger than shared memory: their segments
  int nsegs;
  int pad;
};
// A run of one state's operations applied tile by tile: every operation's
// pairing qubits (dense targets, gadget X/Y qubits) lie in the L tile qubits
// q[0..L-1] (ascending), so each tile of 2^L amplitudes (fixed values of the
// other qubits) goes through shared memory once for the whole run.  L = 0:
// the operations run one by one in global memory.
struct BatchSeg {
  int first_op, nops;    // global operation indices
  int L;
  int pad;
  int8_t q[16];
};
// An operation in its segment's tile coordinates (one per operation, parallel
// to the operation array).
struct BatchXlat {
  uint32_t lctrl, fctrl;    // dense: controls inside the tile (local mask) / outside it (global mask)
  uint32_t lxy, lyz, fyz;   // gadget: local flip and phase masks; phase mask outside the tile (global)
  int nlins;                // dense: number of local insertion positions
  int8_t lins[8];           // dense: ascending local positions of targets and in-tile controls
  int8_t lt[4];             // local target positions (-1: outside the tile, diagonals only)
  int8_t lh;                // gadget: local position of the highest flip bit
};

// Launchers.  Each returns cudaGetLastError() after the launch.  amps is the
// state's device storage, ns its number of storage qubits.
cudaError_t launch_gate1(qs_prec prec, void* amps, const Gate1Params& p, cudaStream_t st);
// SWAP of storage qubits t1 < t2 (qs_gates.cu)
cudaError_t launch_swap(qs_prec prec, void* amps, int ns, int t1, int t2, cudaStream_t st);
cudaError_t launch_dense(qs_prec prec, void* amps, const DenseParams& p, cudaStream_t st);
cudaError_t launch_diag(qs_prec prec, void* amps, const DiagParams& p, cudaStream_t st);
cudaError_t launch_gadget(qs_prec prec, void* amps, const GadgetParams& p, cudaStream_t st);
// complex128 with double-float arithmetic (qs_gates_df.cu)
cudaError_t launch_gate1_df(void* amps, const Gate1DfParams& p, cudaStream_t st);
cudaError_t launch_dense_df(void* amps, const DenseParams& p, cudaStream_t st);
cudaError_t launch_diag_df(void* amps, const DiagParams& p, cudaStream_t st);
cudaError_t launch_gadget_df(void* amps, const GadgetDfParams& p, cudaStream_t st);
// complex128 in block fixed point (qs_gates_fx.cu)
cudaError_t launch_gate1_fx(void* amps, const Gate1FxParams& p, cudaStream_t st);
cudaError_t launch_gate2_fx(void* amps, const Gate2FxParams& p, cudaStream_t st);
cudaError_t launch_diag_fx(void* amps, const DiagFxParams& p, cudaStream_t st);
cudaError_t launch_gadget_fx(void* amps, const GadgetFxParams& p, cudaStream_t st);
// G_DEPOL1, G_DEPOL2, G_DAMP, G_PAULI1
cudaError_t launch_group_fx(void* amps, int op, const GroupFxParams& p, cudaStream_t st);
// complex64 dense gates on the tensor cores, 3 <= n <= 5 (qs_tc.cu)
cudaError_t launch_dense_tc(void* amps, const TcParams& p, cudaStream_t st);
// test of the bounded-wait path: a wait on an mbarrier nothing arrives at, given up after `polls` polls (qs_tc.cu)
cudaError_t launch_test_wait_timeout(int* err, uint32_t polls, cudaStream_t st);
// complex128 dense gates on the bf16 tensor cores, exact integer slices, 3 <= n <= 5 kernel targets (qs_tc_ozaki.cu);
// slices: 7 (49-bit operands, with double-float arithmetic) or 8 (56-bit, with block fixed point)
cudaError_t launch_dense_ozaki(void* amps, const TcParams& p, int slices, cudaStream_t st);
cudaError_t launch_block_compose(const ComposeBlock* blocks, int nblocks, const ComposeInstr* instrs,
                                 const double* data, double* out, cudaStream_t st);
// cost-model network (qs_mlp.cu)
cudaError_t launch_mlp_forward(const float* params, const float* X, const int* idx, int B, float* y, float* z1,
                               float* z2, cudaStream_t st);
cudaError_t launch_mlp_backward(const float* params, const float* X, const float* t, const int* idx, int B,
                                const float* y, const float* z1, const float* z2, float* dy, float* dz1, float* dz2,
                                float* grad, cudaStream_t st);
cudaError_t launch_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr,
                            cudaStream_t st);
int num_sms();  // multiprocessors of the current device (cached)
cudaError_t batch_set_max_smem(int bytes);
cudaError_t launch_batch(qs_prec prec, void* pool, const BatchState* states, const int* order, int nstates,
                         const BatchOp* ops, const double* consts, const BatchSeg* segs, const BatchXlat* xlat,
                         int* counter, int threads, int ctas, int smem_qubits, int wide, cudaStream_t st);
cudaError_t launch_group(qs_prec prec, void* amps, int op, const GroupParams& p, cudaStream_t st);
// complex128 channels in double-float arithmetic: G_DEPOL1, G_DEPOL2, G_DAMP, G_PAULI1 (qs_gates_df.cu)
cudaError_t launch_group_df(void* amps, int op, const GroupParams& p, cudaStream_t st);
cudaError_t launch_ptrace(qs_prec prec, const void* in, void* out, const PtraceParams& p,
                          cudaStream_t st);
cudaError_t launch_superop(const double* kraus, int num_ops, int n, double* sup, cudaStream_t st);
// f64: complex128 in native FP64 (FP64 and block fixed-point arithmetic) instead of double-float
cudaError_t launch_dm_from_pure(qs_prec prec, void* rho, const void* psi, int nq, double weight,
                                int accumulate, cudaStream_t st, bool f64);
cudaError_t launch_init_zero(qs_prec prec, void* amps, int ns, cudaStream_t st);
// bytes (a multiple of 16) from src (device-accessible, 16-byte aligned) to dst
cudaError_t launch_copy16(void* dst, const void* src, size_t bytes, cudaStream_t st);

// Reductions: stage one writes kReduceBlocks complex128 partial sums, stage two
// sums them in a fixed order into result[0] (added to result[0] if accumulate).
// f64: complex128 products and sums in native FP64 (FP64 and block fixed-point
// arithmetic) instead of double-float.
cudaError_t launch_norm(qs_prec prec, const void* amps, int ns, double2* partials, cudaStream_t st, bool f64);
cudaError_t launch_trace(qs_prec prec, const void* amps, int nq, double2* partials, cudaStream_t st);
cudaError_t launch_expec_dm(qs_prec prec, const void* amps, int nq, const PauliTerm* terms,
                            int nterms, double2* partials, cudaStream_t st);
// order: from make_tile_order on the same terms (host copy)
cudaError_t launch_expec_sv(qs_prec prec, const void* amps, int nq, const PauliTerm* terms,
                            int nterms, double2* partials, cudaStream_t st, bool f64, const TileOrder& order);
// the diagonal (I/Z) terms of a statevector Pauli sum by warp Walsh-Hadamard transforms; N >= 5
cudaError_t launch_expec_sv_diag(qs_prec prec, const void* amps, int nq, const PauliTerm* terms, int nterms,
                                 double2* partials, cudaStream_t st, bool f64);
cudaError_t launch_reduce_final(const double2* partials, double2* result, int accumulate, cudaStream_t st,
                                int nblocks = kReduceBlocks);

}  // namespace qsk
