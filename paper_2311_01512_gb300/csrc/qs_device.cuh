// Device-side helpers shared by the kernels: complex types, the bit-insertion
// index core (the paper's Algorithm "bit twiddles"), and block reductions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "qs_internal.h"

namespace qsk {

template <typename R> struct Cplx;
template <> struct Cplx<double> { using T = double2; };
template <> struct Cplx<float> { using T = float2; };

template <typename R>
__device__ __forceinline__ typename Cplx<R>::T mk(R re, R im) {
  typename Cplx<R>::T v;
  v.x = re;
  v.y = im;
  return v;
}

// Insert a zero bit at each sorted position pos[0..n), lowest first
// (insertBits with b = 0): the k-th group's base index.
__device__ __forceinline__ uint64_t insert_zeros(uint64_t k, const int8_t* pos, int n) {
  for (int q = 0; q < n; ++q) {
    const int p = pos[q];
    const uint64_t low = k & ((1ull << p) - 1);
    k = ((k >> p) << (p + 1)) | low;
  }
  return k;
}

__device__ __forceinline__ uint64_t insert_zero(uint64_t k, int p) {
  const uint64_t low = k & ((1ull << p) - 1);
  return ((k >> p) << (p + 1)) | low;
}

// Parity of the set bits of x (the paper's getMaskParity).
__device__ __forceinline__ int parity64(uint64_t x) { return __popcll(x) & 1; }

// Multiply a complex value by i^q.
template <typename T2>
__device__ __forceinline__ T2 rot_i(T2 v, int q) {
  T2 r;
  switch (q & 3) {
    case 0: r = v; break;
    case 1: r.x = -v.y; r.y = v.x; break;
    case 2: r.x = -v.x; r.y = -v.y; break;
    default: r.x = v.y; r.y = -v.x; break;
  }
  return r;
}

// Block-wide sum of a complex128 value; the result is valid in thread 0.
// blockDim.x must be a multiple of 32 and at most 1024.
__device__ __forceinline__ double2 block_sum(double2 v) {
  __shared__ double2 warp_part[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, off);
    v.y += __shfl_down_sync(0xffffffffu, v.y, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_part[warp] = v;
  __syncthreads();
  const int nwarps = blockDim.x >> 5;
  if (warp == 0) {
    v = lane < nwarps ? warp_part[lane] : make_double2(0.0, 0.0);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      v.x += __shfl_down_sync(0xffffffffu, v.x, off);
      v.y += __shfl_down_sync(0xffffffffu, v.y, off);
    }
  }
  return v;
}

// Grid for grid-stride kernels: enough blocks to cover the work, at most
// numSMs x blocks_per_sm.
// Blocks per SM of the grid-stride streaming kernels (one-target gates,
// diagonals, gadgets, channels, SWAP, partial trace): far more than stay
// resident, so that the block scheduler balances the SMs to the end of the
// pass.  Measured at 30 qubits, complex128: 8 per SM left the double-float
// kernels at 85-88% of the HBM copy rate, 48 at 93-98%, 256 at 98-101%.
constexpr int kStreamBlocksPerSM = 256;

inline unsigned grid_for(uint64_t work, int threads, int max_blocks) {
  const uint64_t need = (work + threads - 1) / threads;
  return (unsigned)(need < (uint64_t)max_blocks ? (need == 0 ? 1 : need) : (uint64_t)max_blocks);
}

int num_sms();  // cached cudaDevAttrMultiProcessorCount of the current device

}  // namespace qsk
