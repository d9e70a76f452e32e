// Persistent batched engine: many independent statevectors, each with its own
// circuit, in one launch.  Every CTA repeatedly takes the next state from a
// work counter (states ordered largest first) and applies that state's whole
// program with only block-level synchronisation between operations: in shared
// memory when the state fits, otherwise in place in global memory (small states
// stay in L2).  No CTA ever waits for another one.
//
// Operations (the statevector gates of Sec. "One-target gate", "Many-control
// one-target gate", "Many-target gate", "Phase gadget", "Pauli gadget"):
// dense gates on 1 to 4 targets with controls, diagonals on up to 3 targets,
// Pauli gadgets.  A density matrix is its Choi vector, on which the host has
// lowered unitaries to their two passes and channels to superoperators
// (dense operations on t and t + N).  complex64 states compute in FP32,
// complex128 states in double-float (qs_df.cuh).
#include "qs_device.cuh"
#include "qs_df.cuh"

namespace qsk {

namespace {

using qsdf::df;

// ---- the operation's constants --------------------------------------------
// Converted once per operation from the batch's pool of doubles into shared
// memory (complex64: floats; complex128: double-float pairs), up to 512 reals:
// a 16x16 matrix, 8 diagonal entries, or cos / sin of a gadget.  Converting them per amplitude instead
// would put two f64 -> f32 conversions (FP64 rate) or two integer splits on
// every multiply.
template <typename T2>
struct Konst;
template <>
struct Konst<float2> {
  using K = float;
  __device__ static K conv(double v) { return (float)v; }
};
template <>
struct Konst<double2> {
  using K = df;
  __device__ static K conv(double v) { return qsdf::split(v); }
};

template <typename T2>
using KT = typename Konst<T2>::K;

constexpr int kMaxConsts = 512;

template <typename T2>
__device__ __forceinline__ void load_consts(const BatchOp& op, const double* __restrict__ pool,
                                            typename Konst<T2>::K* kc) {
  const int kind = op.kind;
  const int nreal = kind == 0 ? 2 << (2 * op.n) : (kind == 1 ? 2 << op.n : 2);
  const double* src = pool + op.coff;
  for (int i = threadIdx.x; i < nreal; i += blockDim.x) kc[i] = Konst<T2>::conv(src[i]);
}

// ---- element access -----------------------------------------------------------
// complex64: float2 everywhere.  complex128: double2 in global memory (split
// into double-float pairs on load, rounded to double on store, one DADD per
// real), and in shared memory float4 pairs (re.h, re.l, im.h, im.l), so a state
// or a tile in shared memory goes through all its operations without a split
// or a rounding to double in between.
struct CF {
  float re, im;
};
struct CDF {
  df re, im;
};

__device__ __forceinline__ CF ld(const float2* a, uint32_t i) {
  const float2 v = a[i];
  return CF{v.x, v.y};
}
__device__ __forceinline__ CDF ld(const double2* a, uint32_t i) {
  const double2 v = a[i];
  return CDF{qsdf::split(v.x), qsdf::split(v.y)};
}
__device__ __forceinline__ CDF ld(const float4* a, uint32_t i) {
  const float4 v = a[i];
  return CDF{df{v.x, v.y}, df{v.z, v.w}};
}
__device__ __forceinline__ void st(double2* a, uint32_t i, const qsdf::dot_acc& re, const qsdf::dot_acc& im) {
  a[i] = make_double2(qsdf::finish(re), qsdf::finish(im));
}
__device__ __forceinline__ void st(float4* a, uint32_t i, const qsdf::dot_acc& re, const qsdf::dot_acc& im) {
  const df r = qsdf::dot_result(re), m = qsdf::dot_result(im);
  a[i] = make_float4(r.h, r.l, m.h, m.l);
}

// shared-memory form of a global amplitude and back
template <typename T2>
struct SmemOf;
template <>
struct SmemOf<float2> {
  using T = float2;
  __device__ static T in(float2 v) { return v; }
  __device__ static float2 out(T v) { return v; }
};
template <>
struct SmemOf<double2> {
  using T = float4;
  __device__ static T in(double2 v) {
    const df r = qsdf::split(v.x), m = qsdf::split(v.y);
    return make_float4(r.h, r.l, m.h, m.l);
  }
  __device__ static double2 out(T v) {
    return make_double2(qsdf::to_double(v.x) + qsdf::to_double(v.y), qsdf::to_double(v.z) + qsdf::to_double(v.w));
  }
};

// ---- complex dot products y = sum_k m_k x_k --------------------------------
template <int K>
__device__ __forceinline__ float2 cdot_f32(const float* m, const CF* x) {
  float re = 0.f, im = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float mr = m[2 * k], mi = m[2 * k + 1];
    re = fmaf(mr, x[k].re, re);
    re = fmaf(-mi, x[k].im, re);
    im = fmaf(mr, x[k].im, im);
    im = fmaf(mi, x[k].re, im);
  }
  return make_float2(re, im);
}

template <int K>
__device__ __forceinline__ void cdot_df(const df* m, const CDF* x, qsdf::dot_acc& re, qsdf::dot_acc& im) {
  re = qsdf::dot_first(m[0], x[0].re);
  qsdf::dot_add(re, qsdf::neg(m[1]), x[0].im);
  im = qsdf::dot_first(m[0], x[0].im);
  qsdf::dot_add(im, m[1], x[0].re);
#pragma unroll
  for (int k = 1; k < K; ++k) {
    qsdf::dot_add(re, m[2 * k], x[k].re);
    qsdf::dot_add(re, qsdf::neg(m[2 * k + 1]), x[k].im);
    qsdf::dot_add(im, m[2 * k], x[k].im);
    qsdf::dot_add(im, m[2 * k + 1], x[k].re);
  }
}

// Zero bits inserted at up to 7 ascending positions p_q, given as the masks
// hm_q = ~0 << p_q (unused entries 0): k + (k & hm) shifts the bits at and
// above p up by one and leaves a zero at p.
struct InsMasks {
  uint32_t hm[7];
  int n;
};

__device__ __forceinline__ InsMasks ins_masks(const int8_t* pos, int n) {
  InsMasks m;
  m.n = n;
#pragma unroll
  for (int q = 0; q < 7; ++q) m.hm[q] = q < n ? 0xFFFFFFFFu << pos[q] : 0u;
  return m;
}

__device__ __forceinline__ uint32_t insert_zeros_m(uint32_t k, const InsMasks& m) {
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    if (q >= m.n) break;         // uniform over the block
    k += k & m.hm[q];
  }
  return k;
}

// ---- the arithmetic of one update at given indices ---------------------------
// complex64 (float2, constants as floats)
__device__ __forceinline__ void op_dense1(float2* a, uint32_t i0, uint32_t i1, const float* m) {
  const CF x[2] = {ld(a, i0), ld(a, i1)};
  const float2 y0 = cdot_f32<2>(m, x), y1 = cdot_f32<2>(m + 4, x);
  a[i0] = y0;
  a[i1] = y1;
}
__device__ __forceinline__ void op_dense2(float2* a, const uint32_t* idx, const float* m) {
  CF x[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) x[l] = ld(a, idx[l]);
  float2 y[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) y[j] = cdot_f32<4>(m + 8 * j, x);
#pragma unroll
  for (int j = 0; j < 4; ++j) a[idx[j]] = y[j];
}
// amplitude l of a dense group: base with target bit q set where bit q of l is
template <int NT>
__device__ __forceinline__ uint32_t group_index(uint32_t base, const uint32_t* tb, int l) {
  uint32_t o = base;
#pragma unroll
  for (int q = 0; q < NT; ++q)
    if ((l >> q) & 1) o |= tb[q];
  return o;
}

// dense on the 2^NT amplitudes of the group at base
template <int NT>
__device__ __forceinline__ void op_denseN(float2* a, uint32_t base, const uint32_t* tb, const float* m) {
  constexpr int D = 1 << NT;
  CF x[D];
#pragma unroll
  for (int l = 0; l < D; ++l) x[l] = ld(a, group_index<NT>(base, tb, l));
#pragma unroll
  for (int j = 0; j < D; ++j) a[group_index<NT>(base, tb, j)] = cdot_f32<D>(m + 2 * D * j, x);   // inputs read first
}
__device__ __forceinline__ void op_diag(float2* a, uint32_t i, const float* d) {
  const float2 v = a[i];
  a[i] = make_float2(d[0] * v.x - d[1] * v.y, d[0] * v.y + d[1] * v.x);
}

// complex128 in double-float (P = double2 in global memory, float4 in shared)
template <typename P>
__device__ __forceinline__ void op_dense1(P* a, uint32_t i0, uint32_t i1, const df* m) {
  const CDF x[2] = {ld(a, i0), ld(a, i1)};
  qsdf::dot_acc r0, m0, r1, m1;
  cdot_df<2>(m, x, r0, m0);
  cdot_df<2>(m + 4, x, r1, m1);
  st(a, i0, r0, m0);
  st(a, i1, r1, m1);
}
template <typename P>
__device__ __forceinline__ void op_dense2(P* a, const uint32_t* idx, const df* m) {
  CDF x[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) x[l] = ld(a, idx[l]);
#pragma unroll
  for (int j = 0; j < 4; ++j) {       // every input is read before the first store
    qsdf::dot_acc re, im;
    cdot_df<4>(m + 8 * j, x, re, im);
    st(a, idx[j], re, im);
  }
}
template <int NT, typename P>
__device__ __forceinline__ void op_denseN(P* a, uint32_t base, const uint32_t* tb, const df* m) {
  constexpr int D = 1 << NT;
  CDF x[D];
#pragma unroll
  for (int l = 0; l < D; ++l) x[l] = ld(a, group_index<NT>(base, tb, l));
#pragma unroll
  for (int j = 0; j < D; ++j) {
    qsdf::dot_acc re, im;
    cdot_df<D>(m + 2 * D * j, x, re, im);
    st(a, group_index<NT>(base, tb, j), re, im);
  }
}
template <typename P>
__device__ __forceinline__ void op_diag(P* a, uint32_t i, const df* d) {
  const CDF x = ld(a, i);
  qsdf::dot_acc re, im;
  cdot_df<1>(d, &x, re, im);
  st(a, i, re, im);
}

// Pauli gadget constants: cos(phi), sin(phi), -sin(phi)
template <typename K>
struct Gad {
  K c, s, ns;
};
__device__ __forceinline__ Gad<float> make_gad(const float* kc) { return Gad<float>{kc[0], kc[1], -kc[1]}; }
__device__ __forceinline__ Gad<df> make_gad(const df* kc) { return Gad<df>{kc[0], kc[1], qsdf::neg(kc[1])}; }
// diagonal gadget (no X/Y): a_i -> (c + i s_i) a_i, s_i = -s if neg else s
__device__ __forceinline__ void op_phase(float2* a, uint32_t i, const Gad<float>& G, bool neg) {
  const float si = neg ? G.ns : G.s;
  const float2 v = a[i];
  a[i] = make_float2(G.c * v.x - si * v.y, G.c * v.y + si * v.x);
}
template <typename P>
__device__ __forceinline__ void op_phase(P* a, uint32_t i, const Gad<df>& G, bool neg) {
  const CDF x = ld(a, i);
  const df si = neg ? G.ns : G.s;
  // (c + i si) x: re = c x.re - si x.im, im = c x.im + si x.re
  qsdf::dot_acc re = qsdf::dot_first(G.c, x.re);
  qsdf::dot_add(re, qsdf::neg(si), x.im);
  qsdf::dot_acc im = qsdf::dot_first(G.c, x.im);
  qsdf::dot_add(im, si, x.re);
  st(a, i, re, im);
}
// paired gadget update of (a_i, a_j), j = i xor xy: a_i -> c a_i + s_j i^q a_j and
// a_j -> c a_j + s_i i^q a_i, with s_k = -s where the phase parity of k is odd
__device__ __forceinline__ void op_pair(float2* a, uint32_t i, uint32_t j, const Gad<float>& G, bool negi,
                                        bool negj, int q) {
  const float2 x = a[i], y = a[j];
  const float sj = negj ? G.ns : G.s, si = negi ? G.ns : G.s;
  const float2 ry = rot_i(y, q), rx = rot_i(x, q);
  a[i] = make_float2(G.c * x.x + sj * ry.x, G.c * x.y + sj * ry.y);
  a[j] = make_float2(G.c * y.x + si * rx.x, G.c * y.y + si * rx.y);
}
template <typename P>
__device__ __forceinline__ void op_pair(P* a, uint32_t i, uint32_t j, const Gad<df>& G, bool negi, bool negj,
                                        int q) {
  const CDF x = ld(a, i), y = ld(a, j);
  const df sj = negj ? G.ns : G.s, si = negi ? G.ns : G.s;
  auto rot = [](const CDF& v, int r) {
    switch (r & 3) {
      case 0: return v;
      case 1: return CDF{qsdf::neg(v.im), v.re};
      case 2: return CDF{qsdf::neg(v.re), qsdf::neg(v.im)};
      default: return CDF{v.im, qsdf::neg(v.re)};
    }
  };
  const CDF ry = rot(y, q), rx = rot(x, q);
  qsdf::dot_acc r0 = qsdf::dot_first(G.c, x.re), i0 = qsdf::dot_first(G.c, x.im);
  qsdf::dot_add(r0, sj, ry.re);
  qsdf::dot_add(i0, sj, ry.im);
  qsdf::dot_acc r1 = qsdf::dot_first(G.c, y.re), i1 = qsdf::dot_first(G.c, y.im);
  qsdf::dot_add(r1, si, rx.re);
  qsdf::dot_add(i1, si, rx.im);
  st(a, i, r0, i0);
  st(a, j, r1, i1);
}

// dense sweep on 3 or 4 targets: target bits tb[q] (global or tile-local).
// Out of line, so its registers do not weigh on the other operations.
template <int NT, typename P, typename K>
__device__ __noinline__ void dense_sweep(P* a, uint32_t groups, InsMasks ins, uint32_t ctrl, uint32_t tb0,
                                         uint32_t tb1, uint32_t tb2, uint32_t tb3, const K* kc) {
  const uint32_t tb[4] = {tb0, tb1, tb2, tb3};
  for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x)
    op_denseN<NT>(a, insert_zeros_m(g, ins) | ctrl, tb, kc);
}

// ---- one operation on a whole state held at `a` (shared or global) ---------
// kc: the operation's constants (load_consts).
// WIDE: the batch has dense operations on 3 or 4 targets (superoperators of
// density-matrix channels); without them the kernel carries no call to the
// out-of-line sweeps, whose call sites cost the narrow kernel registers.
template <bool WIDE, typename P, typename K>
__device__ void apply_op(P* a, int nq, const BatchOp& op, const K* kc) {
  const uint32_t dim = 1u << nq;
  const int kind = op.kind, n = op.n;
  if (kind == 0) {
    const int nins = op.nins;
    const InsMasks ins = ins_masks(op.ins, nins);
    const uint32_t ctrl = op.ctrl, b0 = 1u << op.t[0], b1 = n > 1 ? 1u << op.t[1] : 0u;
    const uint32_t groups = dim >> nins;
    if (n == 1) {
      K m[8];   // in registers for the sweep (its stores may alias shared memory)
#pragma unroll
      for (int i = 0; i < 8; ++i) m[i] = kc[i];
      for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x) {
        const uint32_t base = insert_zeros_m(g, ins) | ctrl;
        op_dense1(a, base, base | b0, m);
      }
    } else if (n == 2) {
      for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x) {
        const uint32_t base = insert_zeros_m(g, ins) | ctrl;
        const uint32_t idx[4] = {base, base | b0, base | b1, base | b0 | b1};
        op_dense2(a, idx, kc);
      }
    } else if constexpr (WIDE) {
      const uint32_t tb2 = 1u << op.t[2], tb3 = n > 3 ? 1u << op.t[3] : 0u;
      if (n == 3)
        dense_sweep<3>(a, groups, ins, ctrl, b0, b1, tb2, tb3, kc);
      else
        dense_sweep<4>(a, groups, ins, ctrl, b0, b1, tb2, tb3, kc);
    }
  } else if (kind == 1) {
    const int t0 = op.t[0], t1 = n > 1 ? op.t[1] : 0, t2 = n > 2 ? op.t[2] : 0;
    for (uint32_t i = threadIdx.x; i < dim; i += blockDim.x) {
      int j = (int)((i >> t0) & 1u);
      if (n > 1) j |= (int)((i >> t1) & 1u) << 1;
      if (n > 2) j |= (int)((i >> t2) & 1u) << 2;
      op_diag(a, i, kc + 2 * j);
    }
  } else {
    const auto G = make_gad(kc);
    const uint32_t xy = op.xy, yz = op.yz;
    if (xy == 0) {
      for (uint32_t i = threadIdx.x; i < dim; i += blockDim.x) op_phase(a, i, G, __popc(i & yz) & 1);
    } else {
      const int q = (op.eta + 1) & 3, h = op.h;
      for (uint32_t k = threadIdx.x; k < (dim >> 1); k += blockDim.x) {
        const uint32_t i = ((k >> h) << (h + 1)) | (k & ((1u << h) - 1));
        const uint32_t j = i ^ xy;
        op_pair(a, i, j, G, __popc(i & yz) & 1, __popc(j & yz) & 1, q);
      }
    }
  }
}

// ---- one operation on one tile in shared memory ---------------------------
// Local index i (L bits) is the amplitude base | (i deposited on the tile
// qubits); the translation x gives the operation's masks in local terms and
// the parts outside the tile, which are constant over the tile (taken from
// base).
template <bool WIDE, typename P, typename K>
__device__ void apply_tile_op(P* a, int L, const BatchOp& op, const BatchXlat& x, uint32_t base, const K* kc) {
  const uint32_t dim = 1u << L;
  const int kind = op.kind, n = op.n;
  if (kind == 0) {
    if ((base & x.fctrl) != x.fctrl) return;          // a control outside the tile is 0 here
    const int nins = x.nlins;
    const InsMasks ins = ins_masks(x.lins, nins);
    const uint32_t ctrl = x.lctrl, b0 = 1u << x.lt[0], b1 = n > 1 ? 1u << x.lt[1] : 0u;
    const uint32_t groups = dim >> nins;
    if (n == 1) {
      K m[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) m[i] = kc[i];
      for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x) {
        const uint32_t lb = insert_zeros_m(g, ins) | ctrl;
        op_dense1(a, lb, lb | b0, m);
      }
    } else if (n == 2) {
      for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x) {
        const uint32_t lb = insert_zeros_m(g, ins) | ctrl;
        const uint32_t idx[4] = {lb, lb | b0, lb | b1, lb | b0 | b1};
        op_dense2(a, idx, kc);
      }
    } else if constexpr (WIDE) {
      const uint32_t tb2 = 1u << x.lt[2], tb3 = n > 3 ? 1u << x.lt[3] : 0u;
      if (n == 3)
        dense_sweep<3>(a, groups, ins, ctrl, b0, b1, tb2, tb3, kc);
      else
        dense_sweep<4>(a, groups, ins, ctrl, b0, b1, tb2, tb3, kc);
    }
  } else if (kind == 1) {
    int jfix = 0, lt[3] = {-1, -1, -1};
    for (int q = 0; q < n; ++q) {
      lt[q] = x.lt[q];
      if (lt[q] < 0) jfix |= (int)((base >> op.t[q]) & 1u) << q;
    }
    for (uint32_t i = threadIdx.x; i < dim; i += blockDim.x) {
      int j = jfix;
      if (lt[0] >= 0) j |= (int)((i >> lt[0]) & 1u);
      if (lt[1] >= 0) j |= (int)((i >> lt[1]) & 1u) << 1;
      if (lt[2] >= 0) j |= (int)((i >> lt[2]) & 1u) << 2;
      op_diag(a, i, kc + 2 * j);
    }
  } else {
    const auto G = make_gad(kc);
    const uint32_t fpar = __popc(base & x.fyz) & 1, lyz = x.lyz, lxy = x.lxy;
    if (op.xy == 0) {
      for (uint32_t i = threadIdx.x; i < dim; i += blockDim.x) op_phase(a, i, G, (__popc(i & lyz) & 1) ^ fpar);
    } else {
      const int q = (op.eta + 1) & 3, h = x.lh;
      for (uint32_t k = threadIdx.x; k < (dim >> 1); k += blockDim.x) {
        const uint32_t i = ((k >> h) << (h + 1)) | (k & ((1u << h) - 1));
        const uint32_t j = i ^ lxy;
        op_pair(a, i, j, G, (__popc(i & lyz) & 1) ^ fpar, (__popc(j & lyz) & 1) ^ fpar, q);
      }
    }
  }
}

}  // namespace

// One CTA per state at a time.  States of at most smem_qubits qubits are
// copied to shared memory, run there, and copied back.  Larger states run
// segment by segment: a tiled segment loads each tile (one 16-byte or 8-byte
// gather per amplitude through two 128-entry offset tables; the five lowest
// qubits are always tile qubits, so a warp reads 32 consecutive amplitudes),
// applies the segment's operations to it and writes it back.
template <typename T2, bool WIDE>
__global__ void __launch_bounds__(512, sizeof(T2) == 8 ? 2 : 1)
    k_batch(T2* __restrict__ pool, const BatchState* __restrict__ states, const int* __restrict__ order, int nstates,
            const BatchOp* __restrict__ ops, const double* __restrict__ consts, const BatchSeg* __restrict__ segs,
            const BatchXlat* __restrict__ xlat, int* __restrict__ counter, int smem_qubits) {
  using SM = SmemOf<T2>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typename SM::T* sm = reinterpret_cast<typename SM::T*>(smem_raw);
  __shared__ int s_work;
  __shared__ uint32_t s_tl[128], s_th[128];
  __shared__ KT<T2> s_k[2][kMaxConsts];  // constants of the current and the next operation
  while (true) {
    if (threadIdx.x == 0) s_work = atomicAdd(counter, 1);
    __syncthreads();
    const int w = s_work;
    __syncthreads();
    if (w >= nstates) break;
    const BatchState st = states[order[w]];
    T2* g = pool + st.offset;
    const uint32_t dim = 1u << st.nq;
    if (st.nq <= smem_qubits) {
      for (uint32_t i = threadIdx.x; i < dim; i += blockDim.x) sm[i] = SM::in(g[i]);
      if (st.nops > 0) load_consts<T2>(ops[st.first_op], consts, s_k[0]);
      __syncthreads();
      for (int k = 0; k < st.nops; ++k) {
        apply_op<WIDE>(sm, st.nq, ops[st.first_op + k], s_k[k & 1]);
        if (k + 1 < st.nops) load_consts<T2>(ops[st.first_op + k + 1], consts, s_k[(k + 1) & 1]);
        __syncthreads();
      }
      for (uint32_t i = threadIdx.x; i < dim; i += blockDim.x) g[i] = SM::out(sm[i]);
      __syncthreads();
      continue;
    }
    for (int sg = st.first_seg; sg < st.first_seg + st.nsegs; ++sg) {
      const BatchSeg S = segs[sg];
      if (S.L == 0) {
        load_consts<T2>(ops[S.first_op], consts, s_k[0]);
        __syncthreads();
        for (int k = 0; k < S.nops; ++k) {
          apply_op<WIDE>(g, st.nq, ops[S.first_op + k], s_k[k & 1]);
          if (k + 1 < S.nops) load_consts<T2>(ops[S.first_op + k + 1], consts, s_k[(k + 1) & 1]);
          __syncthreads();
        }
        continue;
      }
      const int L = S.L, hi = L - 7;                  // 8 <= L <= 14
      uint32_t qmask = 0;
      for (int b = 0; b < L; ++b) qmask |= 1u << S.q[b];
      for (int j = threadIdx.x; j < 128; j += blockDim.x) {
        uint32_t tl = 0, th = 0;
        for (int b = 0; b < 7; ++b)
          if ((j >> b) & 1) tl |= 1u << S.q[b];
        for (int b = 0; b < hi; ++b)
          if ((j >> b) & 1) th |= 1u << S.q[7 + b];
        s_tl[j] = tl;
        s_th[j] = th;
      }
      __syncthreads();
      const uint32_t fmask = (dim - 1) & ~qmask;       // the other qubits: the tile number, deposited
      const uint32_t ntiles = dim >> L, tdim = 1u << L;
      for (uint32_t tile = 0; tile < ntiles; ++tile) {
        uint32_t base = 0;
        {
          uint32_t m = fmask, t = tile;
          while (m) {
            const uint32_t low = m & (~m + 1u);
            if (t & 1u) base |= low;
            m ^= low;
            t >>= 1;
          }
        }
        for (uint32_t i = threadIdx.x; i < tdim; i += blockDim.x)
          sm[i] = SM::in(g[base | s_tl[i & 127u] | s_th[i >> 7]]);
        load_consts<T2>(ops[S.first_op], consts, s_k[0]);
        __syncthreads();
        for (int k = 0; k < S.nops; ++k) {
          apply_tile_op<WIDE>(sm, L, ops[S.first_op + k], xlat[S.first_op + k], base, s_k[k & 1]);
          if (k + 1 < S.nops) load_consts<T2>(ops[S.first_op + k + 1], consts, s_k[(k + 1) & 1]);
          __syncthreads();
        }
        for (uint32_t i = threadIdx.x; i < tdim; i += blockDim.x)
          g[base | s_tl[i & 127u] | s_th[i >> 7]] = SM::out(sm[i]);
        __syncthreads();
      }
    }
  }
}

cudaError_t batch_set_max_smem(int bytes) {
  for (const void* f : {(const void*)k_batch<double2, false>, (const void*)k_batch<double2, true>,
                        (const void*)k_batch<float2, false>, (const void*)k_batch<float2, true>}) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// No attribute calls here: this launch is also recorded into a CUDA graph.
cudaError_t launch_batch(qs_prec prec, void* pool, const BatchState* states, const int* order, int nstates,
                         const BatchOp* ops, const double* consts, const BatchSeg* segs, const BatchXlat* xlat,
                         int* counter, int threads, int ctas, int smem_qubits, int wide, cudaStream_t st) {
  const size_t smem = (smem_qubits >= 0 ? (size_t(1) << smem_qubits) : 0) * (prec == QS_C128 ? 16 : 8);
  double2* p128 = static_cast<double2*>(pool);
  float2* p64 = static_cast<float2*>(pool);
  if (prec == QS_C128 && wide)
    k_batch<double2, true><<<ctas, threads, smem, st>>>(p128, states, order, nstates, ops, consts, segs, xlat, counter,
                                                        smem_qubits);
  else if (prec == QS_C128)
    k_batch<double2, false><<<ctas, threads, smem, st>>>(p128, states, order, nstates, ops, consts, segs, xlat,
                                                         counter, smem_qubits);
  else if (wide)
    k_batch<float2, true><<<ctas, threads, smem, st>>>(p64, states, order, nstates, ops, consts, segs, xlat, counter,
                                                       smem_qubits);
  else
    k_batch<float2, false><<<ctas, threads, smem, st>>>(p64, states, order, nstates, ops, consts, segs, xlat, counter,
                                                        smem_qubits);
  return cudaGetLastError();
}

}  // namespace qsk
