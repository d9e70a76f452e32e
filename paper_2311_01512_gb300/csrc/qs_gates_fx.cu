// complex128 kernels in block fixed-point arithmetic (qs_fx.cuh): exact
// integer products, one rounding per output, at least the 53 bits of IEEE
// double.  Same operations and index enumeration as qs_gates.cu and
// qs_density.cu: one- and two-target gates with controls, diagonals, Pauli
// and phase gadgets, and the density-matrix channels that mix amplitudes.
#include "qs_device.cuh"
#include "qs_fx.cuh"

namespace qsk {

using qsfx::Acc;
using qsfx::Part;

namespace {

__device__ __forceinline__ Part part(const FxPart& p) { return Part{p.h, p.l}; }

// the words of a double and its exponent field (hw & 0x7FF00000)
struct Wd {
  uint32_t hw, lw, ef;
};
__device__ __forceinline__ Wd words(double x) {
  Wd w;
  w.hw = (uint32_t)__double2hiint(x);
  w.lw = (uint32_t)__double2loint(x);
  w.ef = w.hw & 0x7FF00000u;
  return w;
}
__device__ __forceinline__ Part fx(const Wd& w, uint32_t exf) { return qsfx::fixed_f(w.hw, w.lw, w.ef, exf); }

struct CPart {
  Part re, im;
};
// a complex amplitude in the block of exponent field exf
__device__ __forceinline__ CPart cfx(const Wd& r, const Wd& i, uint32_t exf) { return CPart{fx(r, exf), fx(i, exf)}; }
__device__ __forceinline__ uint32_t emax2(const Wd& a, const Wd& b) { return max(a.ef, b.ef); }

__device__ __forceinline__ double lin1(Part x, Part f, qsfx::Scale sc) {
  Acc a = qsfx::acc_zero();
  qsfx::mac(a, x, f);
  return qsfx::finish_s(a, sc);
}
__device__ __forceinline__ double lin2(Part x0, Part f0, Part x1, Part f1, qsfx::Scale sc) {
  Acc a = qsfx::acc_zero();
  qsfx::mac(a, x0, f0);
  qsfx::mac(a, x1, f1);
  return qsfx::finish_s(a, sc);
}

// c x for a complex constant c = (re, im, -im parts) and a complex value x
__device__ __forceinline__ double2 cmul(const Part& cr, const Part& ci, const Part& nci, const CPart& x,
                                        qsfx::Scale sc) {
  return make_double2(lin2(x.re, cr, x.im, nci, sc), lin2(x.re, ci, x.im, cr, sc));
}

}  // namespace

// ---------------------------------------------------------------------------
// One-target gate with controls (Sec. "One-target gate", Sec. "Many-control
// one-target gate"): for each pair (i0, i1 = i0 | 2^t), i0 with zero bits
// inserted at the target and control positions and the control bits set,
//   alpha_i0 -> m00 alpha_i0 + m01 alpha_i1,  alpha_i1 -> m10 alpha_i0 + m11 alpha_i1,
// as four real rows over (Re a, Im a, Re b, Im b), the pair sharing one exponent.
// ---------------------------------------------------------------------------
// SINGLE: no controls (one zero bit inserted at t).
template <bool SINGLE>
__global__ void __launch_bounds__(256) k_gate1_fx(double2* __restrict__ psi, const __grid_constant__ Gate1FxParams p) {
  Part m[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) m[r][c] = part(p.m[r][c]);
  const uint64_t tbit = 1ull << p.t;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p.npairs; k += stride) {
    const uint64_t i0 = SINGLE ? insert_zero(k, p.t) : (insert_zeros(k, p.ins, p.nins) | p.ctrl_mask);
    const uint64_t i1 = i0 | tbit;
    const double2 a = psi[i0], b = psi[i1];
    const Wd w[4] = {words(a.x), words(a.y), words(b.x), words(b.y)};
    const uint32_t exf = max(emax2(w[0], w[1]), emax2(w[2], w[3]));
    const Part x[4] = {fx(w[0], exf), fx(w[1], exf), fx(w[2], exf), fx(w[3], exf)};
    const int ex = (int)(exf >> 20);
    const qsfx::Scale sc[2] = {qsfx::scale_for(ex, p.em[0]), qsfx::scale_for(ex, p.em[1])};
    double y[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      Acc acc = qsfx::acc_zero();
#pragma unroll
      for (int c = 0; c < 4; ++c) qsfx::mac(acc, x[c], m[r][c]);
      y[r] = qsfx::finish_s(acc, sc[r >> 1]);
    }
    psi[i0] = make_double2(y[0], y[1]);
    psi[i1] = make_double2(y[2], y[3]);
  }
}

// ---------------------------------------------------------------------------
// Two-target gate with controls (Sec. "Many-target gate", n = 2): for each
// quad i_k = i00 | b0 2^t0 | b1 2^t1 (k = b0 + 2 b1; i00 with zero bits
// inserted at the target and control positions, the control bits set),
//   alpha_{i_j} -> sum_k u_jk alpha_{i_k},
// as eight real rows over the eight parts of the quad, which share one
// exponent; each row sums its eight terms in two accumulators of four
// (qs_fx.cuh).  The constants stay in the parameter space.  Twice the
// one-target gate's integer multiply-adds per amplitude make it bound by the
// integer multipliers (7.75 ms per 30-qubit pass against 5.0 ms for the
// one-target gate), level with the tensor-core form, with the tighter error
// bound of one rounding per output; it also lets a one-qubit unitary or Kraus
// map on a density matrix run as one pass on (t, t + N).
// SINGLE: no controls (two zero bits inserted).
// ---------------------------------------------------------------------------
template <bool SINGLE>
__global__ void __launch_bounds__(256) k_gate2_fx(double2* __restrict__ psi, const __grid_constant__ Gate2FxParams p) {
  const uint64_t b0 = 1ull << p.t0, b1 = 1ull << p.t1;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p.nquads; k += stride) {
    const uint64_t i0 =
        SINGLE ? insert_zero(insert_zero(k, p.lo), p.hi) : (insert_zeros(k, p.ins, p.nins) | p.ctrl_mask);
    const uint64_t idx[4] = {i0, i0 | b0, i0 | b1, i0 | b0 | b1};
    double2 a[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) a[l] = psi[idx[l]];
    Wd w[8];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      w[2 * l] = words(a[l].x);
      w[2 * l + 1] = words(a[l].y);
    }
    uint32_t exf = max(max(emax2(w[0], w[1]), emax2(w[2], w[3])), max(emax2(w[4], w[5]), emax2(w[6], w[7])));
    Part x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fx(w[c], exf);
    const int ex = (int)(exf >> 20);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const qsfx::Scale sc = qsfx::scale_for(ex, p.em[j]);
      double y[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        Acc lo = qsfx::acc_zero(), hi = qsfx::acc_zero();
#pragma unroll
        for (int c = 0; c < 4; ++c) qsfx::mac(lo, x[c], part(p.m[2 * j + u][c]));
#pragma unroll
        for (int c = 4; c < 8; ++c) qsfx::mac(hi, x[c], part(p.m[2 * j + u][c]));
        y[u] = qsfx::finish2_s(lo, hi, sc);
      }
      psi[idx[j]] = make_double2(y[0], y[1]);
    }
  }
}

// ---------------------------------------------------------------------------
// Diagonal: alpha_i -> d_j alpha_i, j = the target bits of i.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(256) k_diag_fx(double2* __restrict__ psi, const __grid_constant__ DiagFxParams p) {
  __shared__ DiagFxEntry d[1 << N];
  for (int j = threadIdx.x; j < (1 << N); j += blockDim.x) d[j] = p.e[j];
  int tp[N];
#pragma unroll
  for (int q = 0; q < N; ++q) tp[q] = p.tpos[q];
  __syncthreads();
  // four amplitudes per iteration (i + u stride, u < 4): their loads are in flight together
  constexpr int U = 4;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.namps; i += U * stride) {
    double2 vs[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t iu = i + u * stride;
      vs[u] = iu < p.namps ? psi[iu] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t iu = i + u * stride;
      if (iu >= p.namps) break;
      const double2 v = vs[u];
      int j = 0;
#pragma unroll
      for (int q = 0; q < N; ++q) j |= (int)((iu >> tp[q]) & 1) << q;
      const Wd wr = words(v.x), wi = words(v.y);
      const uint32_t exf = emax2(wr, wi);
      const DiagFxEntry e = d[j];
      psi[iu] = cmul(part(e.re), part(e.im), part(e.nim), cfx(wr, wi, exf), qsfx::scale_for((int)(exf >> 20), e.em));
    }
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
  const bool pxy = parity64(p.xy & p.yz);     // parity(j & yz) = parity(i & yz) xor this
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p.nwork; k += stride) {
    const uint64_t i = insert_zero(k, p.h);
    const uint64_t j = i ^ p.xy;
    const double2 va = psi[i], vb = psi[j];
    const Wd w[4] = {words(va.x), words(va.y), words(vb.x), words(vb.y)};
    const uint32_t exf = max(emax2(w[0], w[1]), emax2(w[2], w[3]));
    const CPart a = cfx(w[0], w[1], exf), b = cfx(w[2], w[3], exf);
    const qsfx::Scale sc = qsfx::scale_for((int)(exf >> 20), p.em);
    const bool pi = parity64(i & p.yz), pj = pi != pxy;
    // output i: c a + s_j (i^q b)
    const Part bre = odd ? b.im : b.re, bim = odd ? b.re : b.im;
    const Part are = odd ? a.im : a.re, aim = odd ? a.re : a.im;
    const double2 oi = make_double2(lin2(a.re, c, bre, (pj != neg_re) ? ns : s, sc),
                                    lin2(a.im, c, bim, (pj != neg_im) ? ns : s, sc));
    const double2 oj = make_double2(lin2(b.re, c, are, (pi != neg_re) ? ns : s, sc),
                                    lin2(b.im, c, aim, (pi != neg_im) ? ns : s, sc));
    psi[i] = oi;
    psi[j] = oj;
  }
}

// Phase gadget: alpha_i -> (c + i s_i) alpha_i, s_i = -+sin(phi) by parity.
__global__ void __launch_bounds__(256) k_phase_fx(double2* __restrict__ psi, const __grid_constant__ GadgetFxParams p) {
  const Part c = part(p.c), s = part(p.s), ns = part(p.ns);
  // two amplitudes per iteration (i and i + stride): both loads are in flight together
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.nwork; i += 2 * stride) {
    const uint64_t i2 = i + stride;
    const bool has2 = i2 < p.nwork;
    const double2 v0 = psi[i];
    const double2 v1 = has2 ? psi[i2] : make_double2(0.0, 0.0);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint64_t iu = u ? i2 : i;
      if (u && !has2) break;
      const double2 v = u ? v1 : v0;
      const Wd wr = words(v.x), wi = words(v.y);
      const uint32_t exf = emax2(wr, wi);
      const bool odd = parity64(iu & p.yz);
      const Part si = odd ? ns : s, nsi = odd ? s : ns;
      psi[iu] = cmul(c, si, nsi, cfx(wr, wi, exf), qsfx::scale_for((int)(exf >> 20), p.em));
    }
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
      const Wd ar = words(va.x), ai = words(va.y), br = words(vb.x), bi = words(vb.y);
      const Wd cr = words(vc.x), ci = words(vc.y), dr = words(vd.x), di = words(vd.y);
      const uint32_t ead = max(emax2(ar, ai), emax2(dr, di));
      const CPart a = cfx(ar, ai, ead), d = cfx(dr, di, ead);
      const qsfx::Scale s0 = qsfx::scale_for((int)(ead >> 20), p.em[0]);
      if (OP == G_DAMP) {
        rho[i00] = make_double2(lin2(a.re, f[0], d.re, f[1], s0), lin2(a.im, f[0], d.im, f[1], s0));
        const uint32_t ed = emax2(dr, di);
        const CPart dd = cfx(dr, di, ed);
        const qsfx::Scale s3 = qsfx::scale_for((int)(ed >> 20), p.em[3]);
        rho[i11] = make_double2(lin1(dd.re, f[3], s3), lin1(dd.im, f[3], s3));
      } else {
        rho[i00] = make_double2(lin2(a.re, f[0], d.re, f[1], s0), lin2(a.im, f[0], d.im, f[1], s0));
        rho[i11] = make_double2(lin2(d.re, f[0], a.re, f[1], s0), lin2(d.im, f[0], a.im, f[1], s0));
      }
      if (OP == G_PAULI1) {
        const uint32_t ebc = max(emax2(br, bi), emax2(cr, ci));
        const CPart b = cfx(br, bi, ebc), c = cfx(cr, ci, ebc);
        const qsfx::Scale s2 = qsfx::scale_for((int)(ebc >> 20), p.em[2]);
        rho[i01] = make_double2(lin2(b.re, f[2], c.re, f[3], s2), lin2(b.im, f[2], c.im, f[3], s2));
        rho[i10] = make_double2(lin2(c.re, f[2], b.re, f[3], s2), lin2(c.im, f[2], b.im, f[3], s2));
      } else {
        const uint32_t eb = emax2(br, bi), ec = emax2(cr, ci);
        const CPart b = cfx(br, bi, eb), c = cfx(cr, ci, ec);
        const qsfx::Scale sb = qsfx::scale_for((int)(eb >> 20), p.em[2]);
        const qsfx::Scale sc = qsfx::scale_for((int)(ec >> 20), p.em[2]);
        rho[i01] = make_double2(lin1(b.re, f[2], sb), lin1(b.im, f[2], sb));
        rho[i10] = make_double2(lin1(c.re, f[2], sc), lin1(c.im, f[2], sc));
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
      constexpr int mem[4] = {0, 5, 10, 15};
      // the 12 other members, scaled one by one, in three batches of four;
      // each batch is loaded before the stores of the one before it (a load
      // cannot move above a store to the same array)
      constexpr int oth[12] = {1, 2, 3, 4, 6, 7, 8, 9, 11, 12, 13, 14};
      double2 ob[2][4];
      auto scale_batch = [&](const double2* v, int b0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const Wd vr = words(v[u].x), vi = words(v[u].y);
          const uint32_t e = emax2(vr, vi);
          const CPart x = cfx(vr, vi, e);
          const qsfx::Scale se = qsfx::scale_for((int)(e >> 20), p.em[2]);
          rho[idx[oth[b0 + u]]] = make_double2(lin1(x.re, f[2], se), lin1(x.im, f[2], se));
        }
      };
      Wd wr[4], wi[4];
      uint32_t ex = 0;
      double2 dv[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) dv[m] = rho[idx[mem[m]]];
#pragma unroll
      for (int u = 0; u < 4; ++u) ob[0][u] = rho[idx[oth[u]]];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        wr[m] = words(dv[m].x);
        wi[m] = words(dv[m].y);
        ex = max(ex, emax2(wr[m], wi[m]));
      }
      CPart s[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) s[m] = cfx(wr[m], wi[m], ex);
      const qsfx::Scale s0 = qsfx::scale_for((int)(ex >> 20), p.em[0]);
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
        rho[idx[mem[m]]] = make_double2(qsfx::finish_s(re, s0), qsfx::finish_s(im, s0));
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) ob[1][u] = rho[idx[oth[4 + u]]];
      scale_batch(ob[0], 0);
#pragma unroll
      for (int u = 0; u < 4; ++u) ob[0][u] = rho[idx[oth[8 + u]]];
      scale_batch(ob[1], 4);
      scale_batch(ob[0], 8);
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers: grid-stride grids of kStreamBlocksPerSM blocks per SM.
// ---------------------------------------------------------------------------
cudaError_t launch_gate1_fx(void* amps, const Gate1FxParams& p, cudaStream_t st) {
  const unsigned g = grid_for(p.npairs, 256, num_sms() * kStreamBlocksPerSM);
  if (p.nins == 1)
    k_gate1_fx<true><<<g, 256, 0, st>>>(static_cast<double2*>(amps), p);
  else
    k_gate1_fx<false><<<g, 256, 0, st>>>(static_cast<double2*>(amps), p);
  return cudaGetLastError();
}

cudaError_t launch_gate2_fx(void* amps, const Gate2FxParams& p, cudaStream_t st) {
  const unsigned g = grid_for(p.nquads, 256, num_sms() * kStreamBlocksPerSM);
  if (p.nins == 2)
    k_gate2_fx<true><<<g, 256, 0, st>>>(static_cast<double2*>(amps), p);
  else
    k_gate2_fx<false><<<g, 256, 0, st>>>(static_cast<double2*>(amps), p);
  return cudaGetLastError();
}

cudaError_t launch_diag_fx(void* amps, const DiagFxParams& p, cudaStream_t st) {
  const unsigned g = grid_for(p.namps, 256, num_sms() * kStreamBlocksPerSM);
  double2* a = static_cast<double2*>(amps);
  switch (p.n) {
    case 1: k_diag_fx<1><<<g, 256, 0, st>>>(a, p); break;
    case 2: k_diag_fx<2><<<g, 256, 0, st>>>(a, p); break;
    case 3: k_diag_fx<3><<<g, 256, 0, st>>>(a, p); break;
    case 4: k_diag_fx<4><<<g, 256, 0, st>>>(a, p); break;
    case 5: k_diag_fx<5><<<g, 256, 0, st>>>(a, p); break;
    case 6: k_diag_fx<6><<<g, 256, 0, st>>>(a, p); break;
    default: return cudaErrorInvalidValue;
  }
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
