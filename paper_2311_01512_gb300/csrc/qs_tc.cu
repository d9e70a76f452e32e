// Dense n-target gates on the 5th-generation tensor cores (tcgen05) for
// complex64 states: the group update alpha_kj -> sum_l m_jl alpha_kl
// (Sec. "Many-target gate", Eq. (local many-target amplitude update)) is, over
// a tile of 128 groups, the real GEMM
//   C[g, 2j + c] = sum_{l, c'} A[g, 2l + c'] B[2l + c', 2j + c]
// with A the groups' interleaved (re, im) amplitudes and B the realified
// matrix (B[2l, 2j] = Re m_jl, B[2l+1, 2j] = -Im m_jl, B[2l, 2j+1] = Im m_jl,
// B[2l+1, 2j+1] = Re m_jl).  It runs as 3xTF32: A = Ah + Al, B = Bh + Bl with
// Ah, Bh exact TF32 values, C = Ah Bh + Ah Bl + Al Bh accumulated in FP32 in
// tensor memory, which keeps FP32-level accuracy.
//
// One CTA: 256 threads gather a tile through the same bit-insertion
// enumeration as the CUDA-core kernels, split it into TF32 halves and write
// both into shared memory in the UMMA canonical K-major layout (8-row x 16-byte
// core matrices, no swizzle); one thread issues the MMAs and commits them to an
// mbarrier; all eight warps read the accumulator back with tcgen05.ld and
// scatter the results.  Every wait is bounded: on timeout the kernel records
// an error code, frees its tensor memory and returns.
#include "qs_device.cuh"
#include "qs_tc_ptx.cuh"

namespace qsk {
namespace {

using namespace tcptx;

constexpr int kRows = 128;
constexpr uint32_t kWaitLimit = 1u << 26;

}  // namespace

template <int NT>
__global__ void __launch_bounds__(256, 2) k_dense_tc(float2* __restrict__ psi, const __grid_constant__ TcParams p) {
  constexpr int D = 1 << NT;
  constexpr int K = 2 * D;                   // real inputs per group
  constexpr int N = 2 * D;                   // real outputs per group
  constexpr int OPB = kRows * K * 4;         // bytes of one A operand
  constexpr int BPB = N * K * 4;             // bytes of one B operand
  constexpr uint32_t TCOLS = N < 32 ? 32 : N;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* a_hi = smem;
  unsigned char* a_lo = a_hi + OPB;
  unsigned char* b_hi = a_lo + OPB;
  unsigned char* b_lo = b_hi + BPB;
  uint64_t* row_base = reinterpret_cast<uint64_t*>(b_lo + BPB);   // kRows
  uint64_t* toff = row_base + kRows;                               // D
  uint64_t* sc_lo = toff + D;                                      // 32: index bits of e & 31
  uint64_t* sc_hi = sc_lo + 32;                                    // 128: index bits of e >> 5
  uint32_t* gl_lo = reinterpret_cast<uint32_t*>(sc_hi + 128);      // 32: (row | col << 16) bits
  uint32_t* gl_hi = gl_lo + 32;                                    // 128
  uint64_t* mbar = reinterpret_cast<uint64_t*>(gl_hi + 128);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // B = realified matrix, split into TF32 halves, once per CTA.
  for (int e = tid; e < N * K; e += blockDim.x) {
    const int n = e / K, k = e % K;
    const int j = n >> 1, c = n & 1, l = k >> 1, cp = k & 1;
    const double mr = p.mat[2 * (j * D + l)];
    const double mi = p.conj ? -p.mat[2 * (j * D + l) + 1] : p.mat[2 * (j * D + l) + 1];
    const double v = (c == 0) ? (cp == 0 ? mr : -mi) : (cp == 0 ? mi : mr);
    const float f = (float)v;
    const float h = tf32_hi(f);
    const uint32_t off = canon_off(n, k, K);
    *reinterpret_cast<float*>(b_hi + off) = h;
    *reinterpret_cast<float*>(b_lo + off) = f - h;
  }
  for (int j = tid; j < D; j += blockDim.x) {
    uint64_t off = 0;
#pragma unroll
    for (int q = 0; q < NT; ++q)
      if ((j >> q) & 1) off |= 1ull << p.tpos[q];
    toff[j] = off;
  }
  // Tables splitting a tile element e (index order) into its global index
  // bits and its (row, column): row = bits at the free slots of P in order,
  // column l = bits at the target slots (bit q of l at tslot[q]).
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
  const uint32_t idesc = idesc_tf32(kRows, N);
  const uint32_t sbo = K * 32;
  uint32_t phase = 0;
  bool failed = false;

  const int tile = 1 << p.tile_bits;
  const int rows = tile >> NT;
  for (uint64_t c = blockIdx.x; c < p.ntiles && !failed; c += gridDim.x) {
    const uint64_t base = insert_zeros(c, p.hi_ins, p.nhi) | p.ctrl_mask;
    // gather: tile element e (index order) -> row g (free slots), column l (target slots)
    // every load of this thread first, then the shared-memory writes
    constexpr int EPT = kRows * D / 256;
    float2 vals[EPT];
#pragma unroll
    for (int r = 0; r < EPT; ++r) {
      const int e = tid + r * 256;
      if (e < tile) vals[r] = psi[base | sc_lo[e & ((1 << lo_bits) - 1)] | sc_hi[e >> lo_bits]];
    }
#pragma unroll
    for (int r = 0; r < EPT; ++r) {
      const int e = tid + r * 256;
      if (e >= tile) continue;
      const int elo = e & ((1 << lo_bits) - 1), ehi = e >> lo_bits;
      const uint32_t gl = gl_lo[elo] | gl_hi[ehi];
      const int g = (int)(gl & 0xFFFFu), l = (int)(gl >> 16);
      const float2 v = vals[r];
      const float hx = tf32_hi(v.x), hy = tf32_hi(v.y);
      const uint32_t o0 = canon_off(g, 2 * l, K), o1 = canon_off(g, 2 * l + 1, K);
      *reinterpret_cast<float*>(a_hi + o0) = hx;
      *reinterpret_cast<float*>(a_hi + o1) = hy;
      *reinterpret_cast<float*>(a_lo + o0) = v.x - hx;
      *reinterpret_cast<float*>(a_lo + o1) = v.y - hy;
      if (l == 0) row_base[g] = base | sc_lo[elo] | sc_hi[ehi];
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const uint32_t sa_hi = smem_u32(a_hi), sa_lo = smem_u32(a_lo);
      const uint32_t sb_hi = smem_u32(b_hi), sb_lo = smem_u32(b_lo);
      uint32_t acc = 0;
#pragma unroll
      for (int kk = 0; kk < K / 8; ++kk) {     // Al Bh
        mma_tf32(tmem, smem_desc(sa_lo + kk * 256, 128, sbo), smem_desc(sb_hi + kk * 256, 128, sbo), idesc, acc);
        acc = 1;
      }
#pragma unroll
      for (int kk = 0; kk < K / 8; ++kk)       // Ah Bl
        mma_tf32(tmem, smem_desc(sa_hi + kk * 256, 128, sbo), smem_desc(sb_lo + kk * 256, 128, sbo), idesc, 1);
#pragma unroll
      for (int kk = 0; kk < K / 8; ++kk)       // Ah Bh
        mma_tf32(tmem, smem_desc(sa_hi + kk * 256, 128, sbo), smem_desc(sb_hi + kk * 256, 128, sbo), idesc, 1);
      mma_commit(mbar);
    }
    // bounded wait for the MMAs of this tile
    uint32_t spins = 0;
    bool timed_out = false;
    while (!mbar_try_wait(mbar, phase)) {
      if (++spins > kWaitLimit) {
        timed_out = true;
        break;
      }
    }
    phase ^= 1;
    failed = __syncthreads_or(timed_out) != 0;    // the same decision in every thread
    if (failed) {
      if (tid == 0) atomicExch(p.err, 1);
      break;
    }
    fence_after_sync();
    // epilogue: warp w reads lanes 32 (w % 4) .. +31, columns of half (w / 4)
    const int g = 32 * (warp & 3) + lane;
    const int c0 = (warp >> 2) * (N / 2);
    float v[N / 2];
#pragma unroll
    for (int cc = 0; cc < N / 2; cc += 8)
      tmem_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(c0 + cc), v + cc);
    tmem_wait_ld();
    if (g < rows) {
      const uint64_t rb = row_base[g];
#pragma unroll
      for (int cc = 0; cc < N / 2; cc += 2) {
        const int j = (c0 + cc) >> 1;
        psi[rb | toff[j]] = make_float2(v[cc], v[cc + 1]);
      }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
  }
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

template <int NT>
static cudaError_t dense_tc_nt(void* amps, const TcParams& p, cudaStream_t st) {
  constexpr int D = 1 << NT, K = 2 * D, N = 2 * D;
  const size_t smem = 2 * (size_t)kRows * K * 4 + 2 * (size_t)N * K * 4 + 8 * (kRows + D + 160 + 1) + 4 * 160 + 16;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k_dense_tc<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  // CTAs per SM: shared memory (about 200 KiB usable), 8 x 256 threads, and
  // tensor memory (512 columns) all bound it
  int per_sm = (int)((200 * 1024) / smem);
  per_sm = per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm);
  const int tcols = N < 32 ? 32 : N;
  if (per_sm * tcols > 512) per_sm = 512 / tcols;
  const uint64_t maxb = (uint64_t)num_sms() * per_sm;
  const unsigned g = (unsigned)(p.ntiles < maxb ? p.ntiles : maxb);
  k_dense_tc<NT><<<g, 256, smem, st>>>(static_cast<float2*>(amps), p);
  return cudaGetLastError();
}

cudaError_t launch_dense_tc(void* amps, const TcParams& p, cudaStream_t st) {
  switch (p.n) {
    case 3: return dense_tc_nt<3>(amps, p, st);
    case 4: return dense_tc_nt<4>(amps, p, st);
    case 5: return dense_tc_nt<5>(amps, p, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qsk
