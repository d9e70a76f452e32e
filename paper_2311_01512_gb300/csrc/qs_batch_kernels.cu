// Persistent batched engine: many independent statevectors, each with its own
// circuit, in one launch.  Every CTA repeatedly takes the next state from a
// work counter (states ordered largest first) and applies that state's whole
// program with only block-level synchronisation between operations: in shared
// memory when the state fits, otherwise in place in global memory (small states
// stay in L2).  No CTA ever waits for another one.
//
// Operations (the statevector gates of Sec. "One-target gate", "Many-control
// one-target gate", "Many-target gate", "Phase gadget", "Pauli gadget"):
// dense gates on 1 or 2 targets with controls, diagonals on up to 3 targets,
// Pauli gadgets.  complex64 states compute in FP32, complex128 states in
// double-float (qs_df.cuh).
#include "qs_device.cuh"
#include "qs_df.cuh"

namespace qsk {

namespace {

using qsdf::df;

// ---- arithmetic policies -------------------------------------------------
struct ArithF32 {
  using T2 = float2;
  struct C {
    float re, im;
  };
  __device__ static C load(const T2* p) {
    const float2 v = *p;
    return C{v.x, v.y};
  }
  __device__ static void store(T2* p, float re, float im) { *p = make_float2(re, im); }
};

// y = sum_k m_k x_k (complex) over K terms, FP32
template <int K>
__device__ __forceinline__ float2 cdot_f32(const double* m, const ArithF32::C* x) {
  float re = 0.f, im = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float mr = (float)m[2 * k], mi = (float)m[2 * k + 1];
    re = fmaf(mr, x[k].re, re);
    re = fmaf(-mi, x[k].im, re);
    im = fmaf(mr, x[k].im, im);
    im = fmaf(mi, x[k].re, im);
  }
  return make_float2(re, im);
}

struct CDF {
  df re, im;
};

__device__ __forceinline__ CDF load_df(const double2* p) {
  const double2 v = *p;
  return CDF{qsdf::split(v.x), qsdf::split(v.y)};
}

template <int K>
__device__ __forceinline__ double2 cdot_df(const double* m, const CDF* x) {
  CDF c = {qsdf::split(m[0]), qsdf::split(m[1])};
  qsdf::dot_acc re = qsdf::dot_first(c.re, x[0].re);
  qsdf::dot_add(re, qsdf::neg(c.im), x[0].im);
  qsdf::dot_acc im = qsdf::dot_first(c.re, x[0].im);
  qsdf::dot_add(im, c.im, x[0].re);
#pragma unroll
  for (int k = 1; k < K; ++k) {
    c = CDF{qsdf::split(m[2 * k]), qsdf::split(m[2 * k + 1])};
    qsdf::dot_add(re, c.re, x[k].re);
    qsdf::dot_add(re, qsdf::neg(c.im), x[k].im);
    qsdf::dot_add(im, c.re, x[k].im);
    qsdf::dot_add(im, c.im, x[k].re);
  }
  return make_double2(qsdf::finish(re), qsdf::finish(im));
}

__device__ __forceinline__ uint32_t insert_zeros32(uint32_t k, const int8_t* pos, int n) {
  for (int q = 0; q < n; ++q) {
    const int p = pos[q];
    k = ((k >> p) << (p + 1)) | (k & ((1u << p) - 1));
  }
  return k;
}

// ---- one operation on a state held at `a` (shared or global) -------------
template <typename T2>
__device__ void apply_op(T2* a, int nq, const BatchOp& op);

template <>
__device__ void apply_op<float2>(float2* a, int nq, const BatchOp& op) {
  const uint32_t dim = 1u << nq;
  if (op.kind == 0) {
    const int n = op.n;
    const uint32_t groups = dim >> op.nins;
    for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x) {
      const uint32_t base = insert_zeros32(g, op.ins, op.nins) | op.ctrl;
      if (n == 1) {
        const uint32_t i0 = base, i1 = base | (1u << op.t[0]);
        ArithF32::C x[2] = {ArithF32::load(a + i0), ArithF32::load(a + i1)};
        const float2 y0 = cdot_f32<2>(op.m, x), y1 = cdot_f32<2>(op.m + 4, x);
        a[i0] = y0;
        a[i1] = y1;
      } else {
        uint32_t idx[4];
        ArithF32::C x[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          idx[l] = base | ((l & 1) ? (1u << op.t[0]) : 0u) | ((l & 2) ? (1u << op.t[1]) : 0u);
          x[l] = ArithF32::load(a + idx[l]);
        }
        float2 y[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) y[j] = cdot_f32<4>(op.m + 8 * j, x);
#pragma unroll
        for (int j = 0; j < 4; ++j) a[idx[j]] = y[j];
      }
    }
  } else if (op.kind == 1) {
    for (uint32_t i = threadIdx.x; i < dim; i += blockDim.x) {
      int j = 0;
      for (int q = 0; q < op.n; ++q) j |= (int)((i >> op.t[q]) & 1u) << q;
      const float dr = (float)op.m[2 * j], di = (float)op.m[2 * j + 1];
      const float2 v = a[i];
      a[i] = make_float2(dr * v.x - di * v.y, dr * v.y + di * v.x);
    }
  } else {
    const float c = (float)op.c, s = (float)op.s;
    if (op.xy == 0) {
      for (uint32_t i = threadIdx.x; i < dim; i += blockDim.x) {
        const float si = (__popc(i & op.yz) & 1) ? -s : s;
        const float2 v = a[i];
        a[i] = make_float2(c * v.x - si * v.y, c * v.y + si * v.x);
      }
    } else {
      const int q = (op.eta + 1) & 3;
      for (uint32_t k = threadIdx.x; k < (dim >> 1); k += blockDim.x) {
        const uint32_t i = ((k >> op.h) << (op.h + 1)) | (k & ((1u << op.h) - 1));
        const uint32_t j = i ^ op.xy;
        const float2 x = a[i], y = a[j];
        const float sj = (__popc(j & op.yz) & 1) ? -s : s, si = (__popc(i & op.yz) & 1) ? -s : s;
        const float2 ry = rot_i(y, q), rx = rot_i(x, q);
        a[i] = make_float2(c * x.x + sj * ry.x, c * x.y + sj * ry.y);
        a[j] = make_float2(c * y.x + si * rx.x, c * y.y + si * rx.y);
      }
    }
  }
}

template <>
__device__ void apply_op<double2>(double2* a, int nq, const BatchOp& op) {
  const uint32_t dim = 1u << nq;
  if (op.kind == 0) {
    const int n = op.n;
    const uint32_t groups = dim >> op.nins;
    for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x) {
      const uint32_t base = insert_zeros32(g, op.ins, op.nins) | op.ctrl;
      if (n == 1) {
        const uint32_t i0 = base, i1 = base | (1u << op.t[0]);
        CDF x[2] = {load_df(a + i0), load_df(a + i1)};
        const double2 y0 = cdot_df<2>(op.m, x), y1 = cdot_df<2>(op.m + 4, x);
        a[i0] = y0;
        a[i1] = y1;
      } else {
        uint32_t idx[4];
        CDF x[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          idx[l] = base | ((l & 1) ? (1u << op.t[0]) : 0u) | ((l & 2) ? (1u << op.t[1]) : 0u);
          x[l] = load_df(a + idx[l]);
        }
        double2 y[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) y[j] = cdot_df<4>(op.m + 8 * j, x);
#pragma unroll
        for (int j = 0; j < 4; ++j) a[idx[j]] = y[j];
      }
    }
  } else if (op.kind == 1) {
    for (uint32_t i = threadIdx.x; i < dim; i += blockDim.x) {
      int j = 0;
      for (int q = 0; q < op.n; ++q) j |= (int)((i >> op.t[q]) & 1u) << q;
      const CDF x = load_df(a + i);
      a[i] = cdot_df<1>(op.m + 2 * j, &x);
    }
  } else {
    const df c = qsdf::split(op.c), s = qsdf::split(op.s), ns = qsdf::neg(s);
    if (op.xy == 0) {
      for (uint32_t i = threadIdx.x; i < dim; i += blockDim.x) {
        const CDF x = load_df(a + i);
        const df si = (__popc(i & op.yz) & 1) ? ns : s;
        // (c + i si) x: re = c x.re - si x.im, im = c x.im + si x.re
        qsdf::dot_acc re = qsdf::dot_first(c, x.re);
        qsdf::dot_add(re, qsdf::neg(si), x.im);
        qsdf::dot_acc im = qsdf::dot_first(c, x.im);
        qsdf::dot_add(im, si, x.re);
        a[i] = make_double2(qsdf::finish(re), qsdf::finish(im));
      }
    } else {
      const int q = (op.eta + 1) & 3;
      for (uint32_t k = threadIdx.x; k < (dim >> 1); k += blockDim.x) {
        const uint32_t i = ((k >> op.h) << (op.h + 1)) | (k & ((1u << op.h) - 1));
        const uint32_t j = i ^ op.xy;
        const CDF x = load_df(a + i), y = load_df(a + j);
        const df sj = (__popc(j & op.yz) & 1) ? ns : s, si = (__popc(i & op.yz) & 1) ? ns : s;
        auto rot = [](const CDF& v, int r) {
          switch (r & 3) {
            case 0: return v;
            case 1: return CDF{qsdf::neg(v.im), v.re};
            case 2: return CDF{qsdf::neg(v.re), qsdf::neg(v.im)};
            default: return CDF{v.im, qsdf::neg(v.re)};
          }
        };
        const CDF ry = rot(y, q), rx = rot(x, q);
        qsdf::dot_acc r0 = qsdf::dot_first(c, x.re), i0 = qsdf::dot_first(c, x.im);
        qsdf::dot_add(r0, sj, ry.re);
        qsdf::dot_add(i0, sj, ry.im);
        qsdf::dot_acc r1 = qsdf::dot_first(c, y.re), i1 = qsdf::dot_first(c, y.im);
        qsdf::dot_add(r1, si, rx.re);
        qsdf::dot_add(i1, si, rx.im);
        a[i] = make_double2(qsdf::finish(r0), qsdf::finish(i0));
        a[j] = make_double2(qsdf::finish(r1), qsdf::finish(i1));
      }
    }
  }
}

}  // namespace

template <typename T2>
__global__ void k_batch(T2* __restrict__ pool, const BatchState* __restrict__ states, const int* __restrict__ order,
                        int nstates, const BatchOp* __restrict__ ops, int* __restrict__ counter, int smem_qubits) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* sm = reinterpret_cast<T2*>(smem_raw);
  __shared__ int s_work;
  while (true) {
    if (threadIdx.x == 0) s_work = atomicAdd(counter, 1);
    __syncthreads();
    const int w = s_work;
    __syncthreads();
    if (w >= nstates) break;
    const BatchState st = states[order[w]];
    T2* g = pool + st.offset;
    const uint32_t dim = 1u << st.nq;
    const bool in_smem = st.nq <= smem_qubits;
    if (in_smem) {
      for (uint32_t i = threadIdx.x; i < dim; i += blockDim.x) sm[i] = g[i];
      __syncthreads();
    }
    T2* a = in_smem ? sm : g;
    for (int k = 0; k < st.nops; ++k) {
      apply_op<T2>(a, st.nq, ops[st.first_op + k]);
      __syncthreads();
    }
    if (in_smem) {
      for (uint32_t i = threadIdx.x; i < dim; i += blockDim.x) g[i] = sm[i];
      __syncthreads();
    }
  }
}

cudaError_t batch_set_max_smem(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_batch<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_batch<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// No attribute calls here: this launch is also recorded into a CUDA graph.
cudaError_t launch_batch(qs_prec prec, void* pool, const BatchState* states, const int* order, int nstates,
                         const BatchOp* ops, int* counter, int threads, int ctas, int smem_qubits, cudaStream_t st) {
  const size_t smem = (smem_qubits >= 0 ? (size_t(1) << smem_qubits) : 0) * (prec == QS_C128 ? 16 : 8);
  if (prec == QS_C128)
    k_batch<double2><<<ctas, threads, smem, st>>>(static_cast<double2*>(pool), states, order, nstates, ops, counter,
                                                  smem_qubits);
  else
    k_batch<float2><<<ctas, threads, smem, st>>>(static_cast<float2*>(pool), states, order, nstates, ops, counter,
                                                 smem_qubits);
  return cudaGetLastError();
}

}  // namespace qsk
