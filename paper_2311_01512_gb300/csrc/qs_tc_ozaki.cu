// Dense n-target gates (3 <= n <= 5) for complex128 states on the bf16 tensor
// cores, with error-free integer slicing (the Ozaki scheme: Ozaki, Ogita,
// Oishi and Rump, "Error-free transformations of matrix multiplication by
// using fast routines of matrix multiplication and its applications", Numer.
// Algorithms 59 (2012)).
//
// The group update alpha_kj -> sum_l m_jl alpha_kl (Sec. "Many-target gate",
// Eq. (local many-target amplitude update)) over a tile of 128 groups is the
// real GEMM C = A B of k_dense_tc (A: interleaved re/im amplitudes, B: the
// realified matrix).  Every row of A and every column of B is scaled by a
// power of two so that its largest entry lies in [2^48, 2^49], rounded to an
// integer, and cut into seven balanced signed digits (|d_0| <= 129, others
// |d| <= 64):
//   a = 2^(Ea - 6) sum_s a_s 2^(-7 s),   b = 2^(Eb - 6) sum_t b_t 2^(-7 t).
// Digits are exact in bf16; a product of two digit slices summed over
// K <= 64 terms is an integer of at most 2^20, and the sum of the (s, t) slice
// products of one level L = s + t (at most 7 of them) stays below 2^22, so the
// FP32 accumulation in tensor memory is exact.  Levels L = 0..6 are kept (49
// bits; dropped levels are below 2^-48 of the largest term); the epilogue
// recombines them exactly in 64-bit integers, converts once to double and
// applies the row and column scales.  The digits come straight from the FP64
// bit patterns with integer operations (no FP64 arithmetic).
#include "qs_device.cuh"
#include "qs_tc_ptx.cuh"

namespace qsk {
namespace {

using namespace tcptx;

constexpr int kOzRows = 128;
constexpr int kOzSlices = 7;
constexpr uint32_t kOzWaitLimit = 1u << 26;

// Seven bf16 digits of the double with words (hw, lw) relative to the biased
// exponent emax of its row (or column) maximum: V = |x| 2^(48 - Emax) rounded
// to nearest (V <= 2^49), written as V = sum_s d_s 2^(42 - 7s) with balanced
// digits d_1..d_6 in [-64, 63] and d_0 in [0, 129], all multiplied by the
// sign of x.  Balanced digits make the dropped low-order levels symmetric in
// sign, so the truncation carries no bias toward zero.
__device__ __forceinline__ void digits7(uint32_t hw, uint32_t lw, int emax, uint16_t* out) {
  const int eb = (int)((hw >> 20) & 0x7FFu);
  const uint64_t m = ((uint64_t)((hw & 0xFFFFFu) | 0x100000u) << 32) | lw;   // 53-bit significand
  const int shift = emax - eb + 4;                                            // >= 4
  uint64_t v = 0;
  if (eb != 0 && shift < 64) v = (m + (1ull << (shift - 1))) >> shift;
  const uint32_t vh = (uint32_t)(v >> 32), vl = (uint32_t)v;
  int d[kOzSlices];
  int carry = 0;
#pragma unroll
  for (int s = kOzSlices - 1; s >= 1; --s) {
    const int pos = 42 - 7 * s;
    const int u = (int)((pos >= 32 ? (vh >> (pos - 32)) : __funnelshift_r(vl, vh, pos)) & 127u) + carry;
    carry = u >= 64 ? 1 : 0;
    d[s] = u - (carry << 7);
  }
  d[0] = (int)(vh >> 10) + carry;
  const uint32_t sign = hw & 0x80000000u;
#pragma unroll
  for (int s = 0; s < kOzSlices; ++s) {
    const float f = __int_as_float(0x4B400000 + d[s]) - 12582912.0f;   // exact for |d| < 2^22
    out[s] = (uint16_t)((__float_as_uint(f) ^ sign) >> 16);            // bf16 = top half (|d| <= 129)
  }
}

__device__ __forceinline__ int biased_exp(double x) { return (int)(((uint32_t)__double2hiint(x) >> 20) & 0x7FFu); }

// Exact integer value of a level sum (a float holding an integer).  With
// |d_0| <= 129 and |d_s| <= 64 every level is below 2^22 for K <= 64
// (level 0: 64 * 129^2; level L >= 1: 2 * 64 * 129 * 64 + (L - 1) * 64 * 64^2),
// where adding 1.5 * 2^23 exposes the integer in the significand bits.
__device__ __forceinline__ long long level_int(float v) {
  return (long long)(__float_as_int(v + 12582912.0f) - 0x4B400000);
}

}  // namespace

template <int NT, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) k_dense_ozaki(double2* __restrict__ psi, const __grid_constant__ TcParams p) {
  constexpr int D = 1 << NT;
  constexpr int K = 2 * D, N = 2 * D;
  constexpr int ABYTES = kOzRows * K * 2;     // one bf16 digit slice of A
  constexpr int BBYTES = N * K * 2;
  constexpr int EPT = kOzRows * D / THREADS;  // tile elements per thread
  constexpr int CGROUPS = THREADS / 128;      // warps sharing one lane quarter split the columns
  constexpr int CPW = N / CGROUPS;            // accumulator columns per warp (a multiple of 8)
  static_assert(CPW % 8 == 0, "column split");
  constexpr uint32_t TCOLS = (kOzSlices * N) <= 128 ? 128 : ((kOzSlices * N) <= 256 ? 256 : 512);
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* a_dig = smem;                                  // kOzSlices x ABYTES
  unsigned char* b_dig = a_dig + kOzSlices * ABYTES;            // kOzSlices x BBYTES
  uint64_t* row_base = reinterpret_cast<uint64_t*>(b_dig + kOzSlices * BBYTES);  // 128
  uint64_t* toff = row_base + kOzRows;                          // D
  uint64_t* sc_lo = toff + D;                                   // 32
  uint64_t* sc_hi = sc_lo + 32;                                 // 128
  uint32_t* gl_lo = reinterpret_cast<uint32_t*>(sc_hi + 128);   // 32
  uint32_t* gl_hi = gl_lo + 32;                                 // 128
  int* row_exp = reinterpret_cast<int*>(gl_hi + 128);           // 128
  int* col_exp = row_exp + kOzRows;                             // N
  uint64_t* mbar = reinterpret_cast<uint64_t*>(col_exp + N + (N & 1));
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // B: realified matrix, column maxima, digit slices (once per CTA)
  for (int n = tid; n < N; n += blockDim.x) {
    int e = 0;
    for (int k = 0; k < K; ++k) {
      const int j = n >> 1, c = n & 1, l = k >> 1, cp = k & 1;
      const double mr = p.mat[2 * (j * D + l)];
      const double mi = p.conj ? -p.mat[2 * (j * D + l) + 1] : p.mat[2 * (j * D + l) + 1];
      const double v = (c == 0) ? (cp == 0 ? mr : -mi) : (cp == 0 ? mi : mr);
      e = max(e, biased_exp(v));
    }
    col_exp[n] = e;
  }
  __syncthreads();
  for (int idx = tid; idx < N * K; idx += blockDim.x) {
    const int n = idx / K, k = idx % K;
    const int j = n >> 1, c = n & 1, l = k >> 1, cp = k & 1;
    const double mr = p.mat[2 * (j * D + l)];
    const double mi = p.conj ? -p.mat[2 * (j * D + l) + 1] : p.mat[2 * (j * D + l) + 1];
    const double v = (c == 0) ? (cp == 0 ? mr : -mi) : (cp == 0 ? mi : mr);
    uint16_t d[kOzSlices];
    digits7((uint32_t)__double2hiint(v), (uint32_t)__double2loint(v), col_exp[n], d);
    const uint32_t off = canon_off16(n, k, K);
#pragma unroll
    for (int s = 0; s < kOzSlices; ++s) *reinterpret_cast<uint16_t*>(b_dig + s * BBYTES + off) = d[s];
  }
  for (int j = tid; j < D; j += blockDim.x) {
    uint64_t off = 0;
#pragma unroll
    for (int q = 0; q < NT; ++q)
      if ((j >> q) & 1) off |= 1ull << p.tpos[q];
    toff[j] = off;
  }
  const int lo_bits = p.tile_bits < 5 ? p.tile_bits : 5;
  int lo_free = 0;
  for (int b = 0; b < lo_bits; ++b)
    if (!((p.tslot_mask >> b) & 1)) ++lo_free;
  for (int t = tid; t < 32 + 128; t += blockDim.x) {
    const bool lo = t < 32;
    const int v = lo ? t : t - 32;
    const int b0 = lo ? 0 : lo_bits, b1 = lo ? lo_bits : p.tile_bits;
    uint64_t sc = 0;
    uint32_t g = 0, l = 0;
    int gb = lo ? 0 : lo_free;
    for (int b = b0; b < b1; ++b) {
      const uint32_t bit = (uint32_t)(v >> (b - b0)) & 1u;
      sc |= (uint64_t)bit << p.P[b];
      if ((p.tslot_mask >> b) & 1) {
        for (int q = 0; q < NT; ++q)
          if (p.tslot[q] == b) l |= bit << q;
      } else {
        g |= bit << gb;
        ++gb;
      }
    }
    if (lo) {
      sc_lo[v] = sc;
      gl_lo[v] = g | (l << 16);
    } else {
      sc_hi[v] = sc;
      gl_hi[v] = g | (l << 16);
    }
  }
  if (tid == 0) mbar_init(mbar, 1);
  if (warp == 0) {
    tmem_alloc(tmem_slot, TCOLS);
    tmem_relinquish();
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = idesc_bf16(kOzRows, N);
  const uint32_t sbo = K * 16;
  uint32_t phase = 0;
  bool failed = false;
  const int tile = 1 << p.tile_bits;
  const int rows = tile >> NT;

  for (uint64_t c = blockIdx.x; c < p.ntiles && !failed; c += gridDim.x) {
    const uint64_t base = insert_zeros(c, p.hi_ins, p.nhi) | p.ctrl_mask;
    for (int g = tid; g < kOzRows; g += THREADS) row_exp[g] = 0;
    __syncthreads();
    // gather in index order: every load of this thread issued first, then the
    // row maxima of the exponents
    uint32_t w[EPT][4];
#pragma unroll
    for (int r = 0; r < EPT; ++r) {
      const int e = tid + r * THREADS;
      if (e < tile) {
        const double2 v = psi[base | sc_lo[e & ((1 << lo_bits) - 1)] | sc_hi[e >> lo_bits]];
        w[r][0] = (uint32_t)__double2hiint(v.x);
        w[r][1] = (uint32_t)__double2loint(v.x);
        w[r][2] = (uint32_t)__double2hiint(v.y);
        w[r][3] = (uint32_t)__double2loint(v.y);
      }
    }
#pragma unroll
    for (int r = 0; r < EPT; ++r) {
      const int e = tid + r * THREADS;
      if (e >= tile) continue;
      const int elo = e & ((1 << lo_bits) - 1), ehi = e >> lo_bits;
      const uint32_t gl = gl_lo[elo] | gl_hi[ehi];
      const int g = (int)(gl & 0xFFFFu);
      atomicMax(row_exp + g, max((int)((w[r][0] >> 20) & 0x7FFu), (int)((w[r][2] >> 20) & 0x7FFu)));
      if ((gl >> 16) == 0) row_base[g] = base | sc_lo[elo] | sc_hi[ehi];
    }
    __syncthreads();
    // digit slices of A
#pragma unroll
    for (int r = 0; r < EPT; ++r) {
      const int e = tid + r * THREADS;
      if (e >= tile) continue;
      const uint32_t gl = gl_lo[e & ((1 << lo_bits) - 1)] | gl_hi[e >> lo_bits];
      const int g = (int)(gl & 0xFFFFu), l = (int)(gl >> 16);
      const int emax = row_exp[g];
      uint16_t dre[kOzSlices], dim[kOzSlices];
      digits7(w[r][0], w[r][1], emax, dre);
      digits7(w[r][2], w[r][3], emax, dim);
      const uint32_t off = canon_off16(g, 2 * l, K);     // 2l and 2l + 1 share one 4-byte word
#pragma unroll
      for (int s = 0; s < kOzSlices; ++s)
        *reinterpret_cast<uint32_t*>(a_dig + s * ABYTES + off) = (uint32_t)dre[s] | ((uint32_t)dim[s] << 16);
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const uint32_t sa = smem_u32(a_dig), sb = smem_u32(b_dig);
#pragma unroll
      for (int L = 0; L < kOzSlices; ++L) {
        const uint32_t d_tmem = tmem + (uint32_t)(L * N);
        uint32_t acc = 0;
        for (int s = 0; s <= L; ++s) {
          const int t = L - s;
#pragma unroll
          for (int kk = 0; kk < K / 16; ++kk) {
            mma_bf16(d_tmem, smem_desc(sa + s * ABYTES + kk * 256, 128, sbo),
                     smem_desc(sb + t * BBYTES + kk * 256, 128, sbo), idesc, acc);
            acc = 1;
          }
        }
      }
      mma_commit(mbar);
    }
    uint32_t spins = 0;
    bool timed_out = false;
    while (!mbar_try_wait(mbar, phase)) {
      if (++spins > kOzWaitLimit) {
        timed_out = true;
        break;
      }
    }
    phase ^= 1;
    failed = __syncthreads_or(timed_out) != 0;
    if (failed) {
      if (tid == 0) atomicExch(p.err, 1);
      break;
    }
    fence_after_sync();
    // epilogue: lanes 32 (w % 4) .. +31 are rows; warp group (w / 4) takes CPW columns
    const int g = 32 * (warp & 3) + lane;
    const int c0 = (warp >> 2) * CPW;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    const int eg = row_exp[g];
    const uint64_t rb = row_base[g];
#pragma unroll
    for (int cc = 0; cc < CPW; cc += 8) {
      float v[kOzSlices][8];
#pragma unroll
      for (int L = 0; L < kOzSlices; ++L) tmem_ld8(lane_addr + (uint32_t)(L * N + c0 + cc), v[L]);
      tmem_wait_ld();
      if (g < rows) {
        double outv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          long long acc = level_int(v[0][q]);
#pragma unroll
          for (int L = 1; L < kOzSlices; ++L) acc = acc * 128 + level_int(v[L][q]);
          double r = __ll2double_rn(acc);
          // scale 2^(Ea + Eb - 54), Ea, Eb unbiased row / column maximum exponents
          const int scale = eg + col_exp[c0 + cc + q] - 2046 - 54;
          if (acc != 0) r = __hiloint2double(__double2hiint(r) + (int)((unsigned)scale << 20), __double2loint(r));
          outv[q] = r;
        }
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
          const int j = (c0 + cc + q) >> 1;
          psi[rb | toff[j]] = make_double2(outv[q], outv[q + 1]);
        }
      }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
  }
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

template <int NT, int THREADS>
static cudaError_t dense_ozaki_nt(void* amps, const TcParams& p, cudaStream_t st) {
  constexpr int D = 1 << NT, K = 2 * D, N = 2 * D;
  const size_t smem = (size_t)kOzSlices * (kOzRows * K * 2 + N * K * 2) + 8 * (kOzRows + D + 160) + 4 * 160 +
                      4 * (kOzRows + N + 2) + 16 + 64;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e =
        cudaFuncSetAttribute(k_dense_ozaki<NT, THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  constexpr int tcols = (kOzSlices * N) <= 128 ? 128 : ((kOzSlices * N) <= 256 ? 256 : 512);
  int per_sm = (int)((200 * 1024) / smem);
  per_sm = per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm);
  if (per_sm * tcols > 512) per_sm = 512 / tcols;
  const uint64_t maxb = (uint64_t)num_sms() * per_sm;
  const unsigned g = (unsigned)(p.ntiles < maxb ? p.ntiles : maxb);
  k_dense_ozaki<NT, THREADS><<<g, THREADS, smem, st>>>(static_cast<double2*>(amps), p);
  return cudaGetLastError();
}

cudaError_t launch_dense_ozaki(void* amps, const TcParams& p, cudaStream_t st) {
  switch (p.n) {
    case 3: return dense_ozaki_nt<3, 256>(amps, p, st);
    case 4: return dense_ozaki_nt<4, 512>(amps, p, st);
    case 5: return dense_ozaki_nt<5, 512>(amps, p, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qsk
