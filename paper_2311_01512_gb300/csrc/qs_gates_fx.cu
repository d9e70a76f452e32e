// complex128 kernels in block fixed-point arithmetic (qs_fx.cuh): exact
// integer products, one rounding per output, at least the 53 bits of IEEE
// double.  Same operations and index enumeration as qs_gates.cu and
// qs_density.cu: one-target gates with controls, diagonals, Pauli and phase
// gadgets, and the density-matrix channels that mix amplitudes.
#include "qs_device.cuh"
#include "qs_fx.cuh"

namespace qsk {

using qsfx::Acc;
using qsfx::Part;

namespace {

__device__ __forceinline__ Part part(const FxPart& p) { return Part{p.h, p.l}; }

__device__ __forceinline__ uint32_t efield(double x) { return (uint32_t)__double2hiint(x) & 0x7FF00000u; }
__device__ __forceinline__ int ex_of(double2 v) { return (int)(max(efield(v.x), efield(v.y)) >> 20); }
__device__ __forceinline__ int ex_of(double2 a, double2 b) {
  return (int)(max(max(efield(a.x), efield(a.y)), max(efield(b.x), efield(b.y))) >> 20);
}

struct CPart {
  Part re, im;
};
__device__ __forceinline__ CPart cfixed(double2 v, int ex) {
  return CPart{qsfx::fixed_d(v.x, ex), qsfx::fixed_d(v.y, ex)};
}

__device__ __forceinline__ double lin1(Part x, Part f, int ex, int em) {
  Acc a = qsfx::acc_zero();
  qsfx::mac(a, x, f);
  return qsfx::finish(a, ex, em);
}
__device__ __forceinline__ double lin2(Part x0, Part f0, Part x1, Part f1, int ex, int em) {
  Acc a = qsfx::acc_zero();
  qsfx::mac(a, x0, f0);
  qsfx::mac(a, x1, f1);
  return qsfx::finish(a, ex, em);
}

// c x for a complex constant c = (re, im, -im parts) and a complex value x
__device__ __forceinline__ double2 cmul(const Part& cr, const Part& ci, const Part& nci, const CPart& x, int ex, int em) {
  return make_double2(lin2(x.re, cr, x.im, nci, ex, em), lin2(x.re, ci, x.im, cr, ex, em));
}

}  // namespace

// ---------------------------------------------------------------------------
// One-target gate with controls (Sec. "One-target gate", Sec. "Many-control
// one-target gate"): for each pair (i0, i1 = i0 | 2^t), i0 with zero bits
// inserted at the target and control positions and the control bits set,
//   alpha_i0 -> m00 alpha_i0 + m01 alpha_i1,  alpha_i1 -> m10 alpha_i0 + m11 alpha_i1,
// as four real rows over (Re a, Im a, Re b, Im b), the pair sharing one exponent.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gate1_fx(double2* __restrict__ psi, const __grid_constant__ Gate1FxParams p) {
  Part m[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) m[r][c] = part(p.m[r][c]);
  const uint64_t tbit = 1ull << p.t;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p.npairs; k += stride) {
    const uint64_t i0 = insert_zeros(k, p.ins, p.nins) | p.ctrl_mask;
    const uint64_t i1 = i0 | tbit;
    const double2 a = psi[i0], b = psi[i1];
    const int ex = ex_of(a, b);
    const Part x[4] = {qsfx::fixed_d(a.x, ex), qsfx::fixed_d(a.y, ex), qsfx::fixed_d(b.x, ex), qsfx::fixed_d(b.y, ex)};
    double y[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      Acc acc = qsfx::acc_zero();
#pragma unroll
      for (int c = 0; c < 4; ++c) qsfx::mac(acc, x[c], m[r][c]);
      y[r] = qsfx::finish(acc, ex, p.em[r >> 1]);
    }
    psi[i0] = make_double2(y[0], y[1]);
    psi[i1] = make_double2(y[2], y[3]);
  }
}

// ---------------------------------------------------------------------------
// Diagonal: alpha_i -> d_j alpha_i, j = the target bits of i.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_diag_fx(double2* __restrict__ psi, const __grid_constant__ DiagFxParams p) {
  __shared__ DiagFxEntry d[64];
  for (int j = threadIdx.x; j < (1 << p.n); j += blockDim.x) d[j] = p.e[j];
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.namps; i += stride) {
    int j = 0;
    for (int q = 0; q < p.n; ++q) j |= (int)((i >> p.tpos[q]) & 1) << q;
    const double2 v = psi[i];
    const int ex = ex_of(v);
    const DiagFxEntry e = d[j];
    psi[i] = cmul(part(e.re), part(e.im), part(e.nim), cfixed(v, ex), ex, e.em);
  }
}

// ---------------------------------------------------------------------------
// Pauli gadget (Sec. "Pauli gadget"): alpha_i -> c alpha_i + s_j i^q alpha_j,
// j = i xor xy, s_j = -+sin(phi) by the parity of j & yz, q = #Y + 1.  The
// factor i^q permutes and negates the parts of the partner, so each output
// part is c x + (+-s) x' over two parts of the pair.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gadget_fx(double2* __restrict__ psi, const __grid_constant__ GadgetFxParams p) {
  const Part c = part(p.c), s = part(p.s), ns = part(p.ns);
  const int q = (p.eta + 1) & 3;
  // i^q (re, im) = (sr * (odd ? im : re), si * (odd ? re : im))
  const bool odd = q & 1;
  const bool neg_re = q == 1 || q == 2, neg_im = q == 2 || q == 3;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p.nwork; k += stride) {
    const uint64_t i = insert_zero(k, p.h);
    const uint64_t j = i ^ p.xy;
    const double2 va = psi[i], vb = psi[j];
    const int ex = ex_of(va, vb);
    const CPart a = cfixed(va, ex), b = cfixed(vb, ex);
    const bool pj = parity64(j & p.yz), pi = parity64(i & p.yz);
    // output i: c a + s_j (i^q b)
    const Part bre = odd ? b.im : b.re, bim = odd ? b.re : b.im;
    const Part are = odd ? a.im : a.re, aim = odd ? a.re : a.im;
    const double2 oi = make_double2(lin2(a.re, c, bre, (pj != neg_re) ? ns : s, ex, p.em),
                                    lin2(a.im, c, bim, (pj != neg_im) ? ns : s, ex, p.em));
    const double2 oj = make_double2(lin2(b.re, c, are, (pi != neg_re) ? ns : s, ex, p.em),
                                    lin2(b.im, c, aim, (pi != neg_im) ? ns : s, ex, p.em));
    psi[i] = oi;
    psi[j] = oj;
  }
}

// Phase gadget: alpha_i -> (c + i s_i) alpha_i, s_i = -+sin(phi) by parity.
__global__ void __launch_bounds__(256) k_phase_fx(double2* __restrict__ psi, const __grid_constant__ GadgetFxParams p) {
  const Part c = part(p.c), s = part(p.s), ns = part(p.ns);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.nwork; i += stride) {
    const double2 v = psi[i];
    const int ex = ex_of(v);
    const bool odd = parity64(i & p.yz);
    const Part si = odd ? ns : s, nsi = odd ? s : ns;
    psi[i] = cmul(c, si, nsi, cfixed(v, ex), ex, p.em);
  }
}

// ---------------------------------------------------------------------------
// Channels on groups of Choi amplitudes (Sec. "Depolarising channel", Sec.
// "Damping channel", the one-qubit Pauli channel); the updates of k_group in
// qs_density.cu with the coefficients in slots of their own exponent:
//   DEPOL1: 00 <- f0 a + f1 d, 11 <- f0 d + f1 a, 01 <- f2 b, 10 <- f2 c
//           (slots 0, 1 = f0, f1; slot 2 = f2)
//   PAULI1: 00, 11 as DEPOL1; 01 <- f2 b + f3 c, 10 <- f2 c + f3 b
//           (slots 0, 1 = f0, f1; slots 2, 3 = f2, f3)
//   DAMP:   00 <- a + f1 d, 01 <- f2 b, 10 <- f2 c, 11 <- f0 d
//           (slots 0, 1 = 1, f1; slot 2 = f2; slot 3 = f0)
//   DEPOL2: members 0, 5, 10, 15 <- f0 self + f1 (sum of the other three),
//           the other 12 <- f2 self (slots 0, 1 = f0, f1; slot 2 = f2)
// Amplitudes that an output combines share one exponent.
// ---------------------------------------------------------------------------
template <int OP>
__global__ void __launch_bounds__(256) k_group_fx(double2* __restrict__ rho, const __grid_constant__ GroupFxParams p) {
  Part f[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) f[q] = part(p.cf[q]);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p.ngroups; k += stride) {
    const uint64_t base = insert_zeros(k, p.ins, p.nbits);
    if (OP == G_DEPOL1 || OP == G_PAULI1 || OP == G_DAMP) {
      const uint64_t b0 = 1ull << p.mpos[0], b1 = 1ull << p.mpos[1];
      const uint64_t i00 = base, i01 = base | b0, i10 = base | b1, i11 = base | b0 | b1;
      const double2 va = rho[i00], vb = rho[i01], vc = rho[i10], vd = rho[i11];
      const int ead = ex_of(va, vd);
      const CPart a = cfixed(va, ead), d = cfixed(vd, ead);
      if (OP == G_DAMP) {
        rho[i00] = make_double2(lin2(a.re, f[0], d.re, f[1], ead, p.em[0]), lin2(a.im, f[0], d.im, f[1], ead, p.em[0]));
        const int ed = ex_of(vd);
        const CPart dd = cfixed(vd, ed);
        rho[i11] = make_double2(lin1(dd.re, f[3], ed, p.em[3]), lin1(dd.im, f[3], ed, p.em[3]));
      } else {
        rho[i00] = make_double2(lin2(a.re, f[0], d.re, f[1], ead, p.em[0]), lin2(a.im, f[0], d.im, f[1], ead, p.em[0]));
        rho[i11] = make_double2(lin2(d.re, f[0], a.re, f[1], ead, p.em[0]), lin2(d.im, f[0], a.im, f[1], ead, p.em[0]));
      }
      if (OP == G_PAULI1) {
        const int ebc = ex_of(vb, vc);
        const CPart b = cfixed(vb, ebc), c = cfixed(vc, ebc);
        rho[i01] = make_double2(lin2(b.re, f[2], c.re, f[3], ebc, p.em[2]), lin2(b.im, f[2], c.im, f[3], ebc, p.em[2]));
        rho[i10] = make_double2(lin2(c.re, f[2], b.re, f[3], ebc, p.em[2]), lin2(c.im, f[2], b.im, f[3], ebc, p.em[2]));
      } else {
        const int eb = ex_of(vb), ec = ex_of(vc);
        const CPart b = cfixed(vb, eb), c = cfixed(vc, ec);
        rho[i01] = make_double2(lin1(b.re, f[2], eb, p.em[2]), lin1(b.im, f[2], eb, p.em[2]));
        rho[i10] = make_double2(lin1(c.re, f[2], ec, p.em[2]), lin1(c.im, f[2], ec, p.em[2]));
      }
    } else {  // two-qubit depolarising
      uint64_t idx[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        uint64_t v = base;
#pragma unroll
        for (int bb = 0; bb < 4; ++bb)
          if ((m >> bb) & 1) v |= 1ull << p.mpos[bb];
        idx[m] = v;
      }
      const double2 w[4] = {rho[idx[0]], rho[idx[5]], rho[idx[10]], rho[idx[15]]};
      const int ex = max(ex_of(w[0], w[1]), ex_of(w[2], w[3]));
      CPart s[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) s[m] = cfixed(w[m], ex);
      constexpr int mem[4] = {0, 5, 10, 15};
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        Acc re = qsfx::acc_zero(), im = qsfx::acc_zero();
        qsfx::mac(re, s[m].re, f[0]);
        qsfx::mac(im, s[m].im, f[0]);
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          if (o == m) continue;
          qsfx::mac(re, s[o].re, f[1]);
          qsfx::mac(im, s[o].im, f[1]);
        }
        rho[idx[mem[m]]] = make_double2(qsfx::finish(re, ex, p.em[0]), qsfx::finish(im, ex, p.em[0]));
      }
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        if (m == 0 || m == 5 || m == 10 || m == 15) continue;
        const double2 v = rho[idx[m]];
        const int e = ex_of(v);
        const CPart x = cfixed(v, e);
        rho[idx[m]] = make_double2(lin1(x.re, f[2], e, p.em[2]), lin1(x.im, f[2], e, p.em[2]));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers: grid-stride grids of kStreamBlocksPerSM blocks per SM.
// ---------------------------------------------------------------------------
cudaError_t launch_gate1_fx(void* amps, const Gate1FxParams& p, cudaStream_t st) {
  const unsigned g = grid_for(p.npairs, 256, num_sms() * kStreamBlocksPerSM);
  k_gate1_fx<<<g, 256, 0, st>>>(static_cast<double2*>(amps), p);
  return cudaGetLastError();
}

cudaError_t launch_diag_fx(void* amps, const DiagFxParams& p, cudaStream_t st) {
  const unsigned g = grid_for(p.namps, 256, num_sms() * kStreamBlocksPerSM);
  k_diag_fx<<<g, 256, 0, st>>>(static_cast<double2*>(amps), p);
  return cudaGetLastError();
}

cudaError_t launch_gadget_fx(void* amps, const GadgetFxParams& p, cudaStream_t st) {
  const unsigned g = grid_for(p.nwork, 256, num_sms() * kStreamBlocksPerSM);
  if (p.xy == 0)
    k_phase_fx<<<g, 256, 0, st>>>(static_cast<double2*>(amps), p);
  else
    k_gadget_fx<<<g, 256, 0, st>>>(static_cast<double2*>(amps), p);
  return cudaGetLastError();
}

cudaError_t launch_group_fx(void* amps, int op, const GroupFxParams& p, cudaStream_t st) {
  double2* a = static_cast<double2*>(amps);
  const unsigned g = grid_for(p.ngroups, 256, num_sms() * kStreamBlocksPerSM);
  switch (op) {
    case G_DEPOL1: k_group_fx<G_DEPOL1><<<g, 256, 0, st>>>(a, p); break;
    case G_DEPOL2: k_group_fx<G_DEPOL2><<<g, 256, 0, st>>>(a, p); break;
    case G_DAMP: k_group_fx<G_DAMP><<<g, 256, 0, st>>>(a, p); break;
    case G_PAULI1: k_group_fx<G_PAULI1><<<g, 256, 0, st>>>(a, p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace qsk
