// complex128 unitary-type kernels with double-float arithmetic on the FP32
// pipes (qs_df.cuh).  Same operations and index enumeration as qs_gates.cu:
// one-target gates, dense many-target gates, diagonals, Pauli / phase gadgets.
#include "qs_device.cuh"
#include "qs_df.cuh"

namespace qsk {

using qsdf::df;

struct cdf {
  df re, im;
};

__device__ __forceinline__ cdf load_split(const double2* p) {
  const double2 v = *p;
  cdf r;
  r.re = qsdf::split(v.x);
  r.im = qsdf::split(v.y);
  return r;
}

__device__ __forceinline__ double2 join2(df re, df im) { return make_double2(qsdf::join(re), qsdf::join(im)); }

// c * x for complex df constant c and complex df value x, accumulated as two
// real dot products: re += c.re x.re - c.im x.im, im += c.re x.im + c.im x.re.
struct cacc {
  qsdf::dot_acc re, im;
};

__device__ __forceinline__ cacc cmul_first(const cdf& c, const cdf& x) {
  cacc a;
  a.re = qsdf::dot_first(c.re, x.re);
  qsdf::dot_add(a.re, qsdf::neg(c.im), x.im);
  a.im = qsdf::dot_first(c.re, x.im);
  qsdf::dot_add(a.im, c.im, x.re);
  return a;
}

__device__ __forceinline__ void cmul_add(cacc& a, const cdf& c, const cdf& x) {
  qsdf::dot_add(a.re, c.re, x.re);
  qsdf::dot_add(a.re, qsdf::neg(c.im), x.im);
  qsdf::dot_add(a.im, c.re, x.im);
  qsdf::dot_add(a.im, c.im, x.re);
}

__device__ __forceinline__ double2 cacc_result(const cacc& a) {
  return make_double2(qsdf::finish(a.re), qsdf::finish(a.im));
}

// ---------------------------------------------------------------------------
// One-target gate (Sec. "One-target gate", "Many-control one-target gate").
// Chunks of 32 consecutive pairs (one warp) with (chunk mod f64_mod) <
// f64_count run in native FP64 instead, so that the FP64 pipe, idle otherwise,
// takes a share of the work; the choice is warp-uniform.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 6) k_gate1_df(double2* __restrict__ psi, const __grid_constant__ Gate1DfParams p) {
  cdf m[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    m[e].re = df{p.mh[2 * e], p.ml[2 * e]};
    m[e].im = df{p.mh[2 * e + 1], p.ml[2 * e + 1]};
  }
  const uint64_t tbit = 1ull << p.t;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p.f64_count == 0) {
    // two pairs per iteration: all four loads issued before the arithmetic
    for (; k + stride < p.npairs; k += 2 * stride) {
      const uint64_t i0 = insert_zeros(k, p.ins, p.nins) | p.ctrl_mask;
      const uint64_t j0 = insert_zeros(k + stride, p.ins, p.nins) | p.ctrl_mask;
      const double2 a2 = psi[i0], b2 = psi[i0 | tbit], c2 = psi[j0], d2 = psi[j0 | tbit];
      cdf a, b;
      a.re = qsdf::split(a2.x); a.im = qsdf::split(a2.y);
      b.re = qsdf::split(b2.x); b.im = qsdf::split(b2.y);
      cacc r0 = cmul_first(m[0], a);
      cmul_add(r0, m[1], b);
      cacc r1 = cmul_first(m[2], a);
      cmul_add(r1, m[3], b);
      psi[i0] = cacc_result(r0);
      psi[i0 | tbit] = cacc_result(r1);
      a.re = qsdf::split(c2.x); a.im = qsdf::split(c2.y);
      b.re = qsdf::split(d2.x); b.im = qsdf::split(d2.y);
      r0 = cmul_first(m[0], a);
      cmul_add(r0, m[1], b);
      r1 = cmul_first(m[2], a);
      cmul_add(r1, m[3], b);
      psi[j0] = cacc_result(r0);
      psi[j0 | tbit] = cacc_result(r1);
    }
  }
  for (; k < p.npairs; k += stride) {
    const uint64_t i0 = insert_zeros(k, p.ins, p.nins) | p.ctrl_mask;
    const uint64_t i1 = i0 | tbit;
    const uint32_t chunk = (uint32_t)(k >> 5);
    if (p.f64_count > 0 && (int)(chunk % (uint32_t)p.f64_mod) < p.f64_count) {
      const double2 a = psi[i0], b = psi[i1];
      double2 r0, r1;
      r0.x = p.m[0] * a.x - p.m[1] * a.y + p.m[2] * b.x - p.m[3] * b.y;
      r0.y = p.m[0] * a.y + p.m[1] * a.x + p.m[2] * b.y + p.m[3] * b.x;
      r1.x = p.m[4] * a.x - p.m[5] * a.y + p.m[6] * b.x - p.m[7] * b.y;
      r1.y = p.m[4] * a.y + p.m[5] * a.x + p.m[6] * b.y + p.m[7] * b.x;
      psi[i0] = r0;
      psi[i1] = r1;
    } else {
      const cdf a = load_split(psi + i0), b = load_split(psi + i1);
      cacc r0 = cmul_first(m[0], a);
      cmul_add(r0, m[1], b);
      cacc r1 = cmul_first(m[2], a);
      cmul_add(r1, m[3], b);
      psi[i0] = cacc_result(r0);
      psi[i1] = cacc_result(r1);
    }
  }
}

// ---------------------------------------------------------------------------
// Dense n-target gate (Sec. "Many-target gate"), tiled exactly as k_dense; the
// tile holds split amplitudes (two float pairs, 16 bytes, as a double2 would).
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(256) k_dense_df(double2* __restrict__ psi, const __grid_constant__ DenseParams p) {
  constexpr int D = 1 << NT;
  constexpr int kTile = 1 << kTileBits;
  constexpr int EPT = kTile / 256;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cdf* sm_mat = reinterpret_cast<cdf*>(smem_raw);          // D x D
  cdf* sm_tile = sm_mat + D * D;                            // up to kTile
  uint32_t* sm_toff = reinterpret_cast<uint32_t*>(sm_tile + kTile);

  for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
    const double re = p.mat[2 * e];
    const double im = p.conj ? -p.mat[2 * e + 1] : p.mat[2 * e + 1];
    cdf v;
    v.re = qsdf::split(re);
    v.im = qsdf::split(im);
    sm_mat[e] = v;
  }
  for (int l = threadIdx.x; l < D; l += blockDim.x) {
    uint32_t off = 0;
#pragma unroll
    for (int q = 0; q < NT; ++q) off |= ((uint32_t)(l >> q) & 1u) << p.tslot[q];
    sm_toff[l] = off;
  }
  uint32_t tslot_mask = 0;
#pragma unroll
  for (int q = 0; q < NT; ++q) tslot_mask |= 1u << p.tslot[q];
  const int tile = 1 << p.tile_bits;
  __syncthreads();

  for (uint64_t c = blockIdx.x; c < p.ntiles; c += gridDim.x) {
    const uint64_t base = insert_zeros(c, p.hi_ins, p.nhi) | p.ctrl_mask;
    uint64_t gidx[EPT];
#pragma unroll
    for (int r = 0; r < EPT; ++r) {
      const int e = threadIdx.x + r * 256;
      uint64_t idx = base;
      for (int b = 0; b < p.tile_bits; ++b) idx |= (uint64_t)((e >> b) & 1) << p.P[b];
      gidx[r] = idx;
      if (e < tile) sm_tile[e] = load_split(psi + idx);
    }
    __syncthreads();
    double2 out[EPT];
#pragma unroll
    for (int r = 0; r < EPT; ++r) {
      const int e = threadIdx.x + r * 256;
      out[r] = make_double2(0.0, 0.0);
      if (e < tile) {
        int j = 0;
#pragma unroll
        for (int q = 0; q < NT; ++q) j |= ((e >> p.tslot[q]) & 1) << q;
        const uint32_t e0 = (uint32_t)e & ~tslot_mask;
        const cdf* mrow = sm_mat + j * D;
        cacc acc = cmul_first(mrow[0], sm_tile[e0 | sm_toff[0]]);
#pragma unroll 4
        for (int l = 1; l < D; ++l) cmul_add(acc, mrow[l], sm_tile[e0 | sm_toff[l]]);
        out[r] = cacc_result(acc);
      }
    }
#pragma unroll
    for (int r = 0; r < EPT; ++r) {
      const int e = threadIdx.x + r * 256;
      if (e < tile) psi[gidx[r]] = out[r];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Diagonal: alpha_i -> d_j alpha_i.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int diag_index(uint64_t i, const DiagParams& p) {
  int j = 0;
  for (int q = 0; q < p.n; ++q) j |= (int)((i >> p.tpos[q]) & 1) << q;
  return j;
}

__global__ void __launch_bounds__(256, 8) k_diag_df(double2* __restrict__ psi, const __grid_constant__ DiagParams p) {
  __shared__ cdf d[64];
  for (int j = threadIdx.x; j < (1 << p.n); j += blockDim.x) {
    cdf v;
    v.re = qsdf::split(p.d[2 * j]);
    v.im = qsdf::split(p.d[2 * j + 1]);
    d[j] = v;
  }
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // two amplitudes per iteration, both loads issued first
  for (; i + stride < p.namps; i += 2 * stride) {
    const double2 v0 = psi[i], v1 = psi[i + stride];
    cdf a;
    a.re = qsdf::split(v0.x);
    a.im = qsdf::split(v0.y);
    psi[i] = cacc_result(cmul_first(d[diag_index(i, p)], a));
    a.re = qsdf::split(v1.x);
    a.im = qsdf::split(v1.y);
    psi[i + stride] = cacc_result(cmul_first(d[diag_index(i + stride, p)], a));
  }
  for (; i < p.namps; i += stride) {
    const cdf a = load_split(psi + i);
    psi[i] = cacc_result(cmul_first(d[diag_index(i, p)], a));
  }
}

// ---------------------------------------------------------------------------
// Pauli gadget (Sec. "Pauli gadget"): alpha_i -> c alpha_i + s_j (i^q alpha_j),
// s_j = +-sin(phi) by the parity of j & yz, q = #Y + 1; the multiplication by
// i^q is an exact permutation and negation of the split parts.
// ---------------------------------------------------------------------------
__device__ __forceinline__ cdf rot_cdf(const cdf& v, int q) {
  cdf r;
  switch (q & 3) {
    case 0: r = v; break;
    case 1: r.re = qsdf::neg(v.im); r.im = v.re; break;
    case 2: r.re = qsdf::neg(v.re); r.im = qsdf::neg(v.im); break;
    default: r.re = v.im; r.im = qsdf::neg(v.re); break;
  }
  return r;
}

__device__ __forceinline__ double2 lin2(df c, const cdf& a, df s, const cdf& b) {
  qsdf::dot_acc re = qsdf::dot_first(c, a.re);
  qsdf::dot_add(re, s, b.re);
  qsdf::dot_acc im = qsdf::dot_first(c, a.im);
  qsdf::dot_add(im, s, b.im);
  return make_double2(qsdf::finish(re), qsdf::finish(im));
}

__global__ void __launch_bounds__(256, 8) k_gadget_df(double2* __restrict__ psi, const __grid_constant__ GadgetDfParams p) {
  const df c{p.ch, p.cl}, s{p.sh, p.sl}, ns{-p.sh, -p.sl};
  const int q = (p.eta + 1) & 3;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p.nwork; k += stride) {
    const uint64_t i = insert_zero(k, p.h);
    const uint64_t j = i ^ p.xy;
    const cdf a = load_split(psi + i), b = load_split(psi + j);
    const df sj = parity64(j & p.yz) ? ns : s;
    const df si = parity64(i & p.yz) ? ns : s;
    psi[i] = lin2(c, a, sj, rot_cdf(b, q));
    psi[j] = lin2(c, b, si, rot_cdf(a, q));
  }
}

// Phase gadget: alpha_i -> (c + i s_i) alpha_i.
__global__ void __launch_bounds__(256, 8) k_phase_df(double2* __restrict__ psi, const __grid_constant__ GadgetDfParams p) {
  const df c{p.ch, p.cl}, s{p.sh, p.sl}, ns{-p.sh, -p.sl};
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + stride < p.nwork; i += 2 * stride) {
    const double2 v0 = psi[i], v1 = psi[i + stride];
    cdf a;
    a.re = qsdf::split(v0.x);
    a.im = qsdf::split(v0.y);
    psi[i] = lin2(c, a, parity64(i & p.yz) ? ns : s, rot_cdf(a, 1));
    a.re = qsdf::split(v1.x);
    a.im = qsdf::split(v1.y);
    psi[i + stride] = lin2(c, a, parity64((i + stride) & p.yz) ? ns : s, rot_cdf(a, 1));
  }
  for (; i < p.nwork; i += stride) {
    const cdf a = load_split(psi + i);
    const df si = parity64(i & p.yz) ? ns : s;
    psi[i] = lin2(c, a, si, rot_cdf(a, 1));
  }
}

// ---------------------------------------------------------------------------
// Channels on groups of Choi amplitudes, double-float arithmetic.  The same
// updates as k_group in qs_density.cu (Sec. "Depolarising channel", "Damping
// channel"; the one-qubit Pauli channel): each output is a real combination
// of at most four amplitudes of its group, formed as an error-free FP32 dot
// product and rounded once to double.  (Dephasing only scales and stays on
// the FP64 kernel, which already moves memory at the HBM rate.)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 lin_df(df ca, const cdf& x, df cb, const cdf& y) {
  qsdf::dot_acc re = qsdf::dot_first(ca, x.re), im = qsdf::dot_first(ca, x.im);
  qsdf::dot_add(re, cb, y.re);
  qsdf::dot_add(im, cb, y.im);
  return make_double2(qsdf::finish(re), qsdf::finish(im));
}

__device__ __forceinline__ double2 scale_df(df c, const cdf& x) {
  return make_double2(qsdf::finish(qsdf::dot_first(c, x.re)), qsdf::finish(qsdf::dot_first(c, x.im)));
}

__device__ __forceinline__ cdf split2(double2 v) {
  cdf r;
  r.re = qsdf::split(v.x);
  r.im = qsdf::split(v.y);
  return r;
}

template <int OP>
__global__ void __launch_bounds__(256) k_group_df(double2* __restrict__ rho, const __grid_constant__ GroupParams p) {
  const df f0 = qsdf::split(p.f[0]), f1 = qsdf::split(p.f[1]), f2 = qsdf::split(p.f[2]), f3 = qsdf::split(p.f[3]);
  const df one{1.0f, 0.0f};
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p.ngroups; k += stride) {
    const uint64_t base = insert_zeros(k, p.ins, p.nbits);
    if (OP == G_DEPOL1 || OP == G_PAULI1 || OP == G_DAMP) {
      const uint64_t b0 = 1ull << p.mpos[0], b1 = 1ull << p.mpos[1];
      const uint64_t i00 = base, i01 = base | b0, i10 = base | b1, i11 = base | b0 | b1;
      const double2 va = rho[i00], vb = rho[i01], vc = rho[i10], vd = rho[i11];
      const cdf a = split2(va), b = split2(vb), c = split2(vc), d = split2(vd);
      if (OP == G_DEPOL1) {
        rho[i00] = lin_df(f0, a, f1, d);
        rho[i11] = lin_df(f0, d, f1, a);
        rho[i01] = scale_df(f2, b);
        rho[i10] = scale_df(f2, c);
      } else if (OP == G_PAULI1) {
        rho[i00] = lin_df(f0, a, f1, d);
        rho[i11] = lin_df(f0, d, f1, a);
        rho[i01] = lin_df(f2, b, f3, c);
        rho[i10] = lin_df(f2, c, f3, b);
      } else {  // damping
        rho[i00] = lin_df(one, a, f1, d);
        rho[i01] = scale_df(f2, b);
        rho[i10] = scale_df(f2, c);
        rho[i11] = scale_df(f0, d);
      }
    } else {  // two-qubit depolarising: members 0, 5, 10, 15 mix, the other 12 scale
      uint64_t idx[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        uint64_t v = base;
#pragma unroll
        for (int bb = 0; bb < 4; ++bb)
          if ((m >> bb) & 1) v |= 1ull << p.mpos[bb];
        idx[m] = v;
      }
      const double2 w0 = rho[idx[0]], w5 = rho[idx[5]], w10 = rho[idx[10]], w15 = rho[idx[15]];
      const cdf s[4] = {split2(w0), split2(w5), split2(w10), split2(w15)};
      constexpr int mem[4] = {0, 5, 10, 15};
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        qsdf::dot_acc re = qsdf::dot_first(f0, s[m].re), im = qsdf::dot_first(f0, s[m].im);
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          if (o == m) continue;
          qsdf::dot_add(re, f1, s[o].re);
          qsdf::dot_add(im, f1, s[o].im);
        }
        rho[idx[mem[m]]] = make_double2(qsdf::finish(re), qsdf::finish(im));
      }
      constexpr int oth[12] = {1, 2, 3, 4, 6, 7, 8, 9, 11, 12, 13, 14};
#pragma unroll
      for (int b0 = 0; b0 < 12; b0 += 6) {            // loads of a batch before its stores
        double2 x[6];
#pragma unroll
        for (int u = 0; u < 6; ++u) x[u] = rho[idx[oth[b0 + u]]];
#pragma unroll
        for (int u = 0; u < 6; ++u) rho[idx[oth[b0 + u]]] = scale_df(f2, split2(x[u]));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_group_df(void* amps, int op, const GroupParams& p, cudaStream_t st) {
  double2* a = static_cast<double2*>(amps);
  const unsigned g = grid_for(p.ngroups, 256, num_sms() * kStreamBlocksPerSM);
  switch (op) {
    case G_DEPOL1: k_group_df<G_DEPOL1><<<g, 256, 0, st>>>(a, p); break;
    case G_DEPOL2: k_group_df<G_DEPOL2><<<g, 256, 0, st>>>(a, p); break;
    case G_DAMP: k_group_df<G_DAMP><<<g, 256, 0, st>>>(a, p); break;
    case G_PAULI1: k_group_df<G_PAULI1><<<g, 256, 0, st>>>(a, p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
cudaError_t launch_gate1_df(void* amps, const Gate1DfParams& p, cudaStream_t st) {
  const unsigned g = grid_for(p.npairs, 256, num_sms() * kStreamBlocksPerSM);
  k_gate1_df<<<g, 256, 0, st>>>(static_cast<double2*>(amps), p);
  return cudaGetLastError();
}

template <int NT>
static cudaError_t dense_df_nt(void* amps, const DenseParams& p, cudaStream_t st) {
  constexpr int D = 1 << NT;
  const size_t smem = sizeof(cdf) * (D * D + (1 << kTileBits)) + sizeof(uint32_t) * D;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k_dense_df<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  const int per_sm = smem > 100 * 1024 ? 1 : (smem > 60 * 1024 ? 2 : 4);
  const uint64_t maxb = (uint64_t)num_sms() * per_sm;
  const unsigned g = (unsigned)(p.ntiles < maxb ? p.ntiles : maxb);
  k_dense_df<NT><<<g, 256, smem, st>>>(static_cast<double2*>(amps), p);
  return cudaGetLastError();
}

cudaError_t launch_dense_df(void* amps, const DenseParams& p, cudaStream_t st) {
  switch (p.n) {
    case 1: return dense_df_nt<1>(amps, p, st);
    case 2: return dense_df_nt<2>(amps, p, st);
    case 3: return dense_df_nt<3>(amps, p, st);
    case 4: return dense_df_nt<4>(amps, p, st);
    case 5: return dense_df_nt<5>(amps, p, st);
    case 6: return dense_df_nt<6>(amps, p, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_diag_df(void* amps, const DiagParams& p, cudaStream_t st) {
  const unsigned g = grid_for(p.namps, 256, num_sms() * kStreamBlocksPerSM);
  k_diag_df<<<g, 256, 0, st>>>(static_cast<double2*>(amps), p);
  return cudaGetLastError();
}

cudaError_t launch_gadget_df(void* amps, const GadgetDfParams& p, cudaStream_t st) {
  const unsigned g = grid_for(p.nwork, 256, num_sms() * kStreamBlocksPerSM);
  if (p.xy == 0)
    k_phase_df<<<g, 256, 0, st>>>(static_cast<double2*>(amps), p);
  else
    k_gadget_df<<<g, 256, 0, st>>>(static_cast<double2*>(amps), p);
  return cudaGetLastError();
}

}  // namespace qsk
