// lc_group.cuh — thread-group layouts of the degree-binned vertex kernels.
#pragma once

#include "lc_internal.cuh"

namespace lc {

// ---------------------------------------------------------------- groups

// GS threads per vertex.  GS <= 32: aligned lane groups inside a warp;
// GS > 32: the whole block (blockDim.x == GS).
template <int GS>
struct Grp {
  static constexpr bool kWarp = GS <= 32;
  static constexpr int kWarps = GS > 32 ? GS / 32 : 1;

  __device__ static int rank() { return kWarp ? (int)(threadIdx.x & (GS - 1)) : (int)threadIdx.x; }

  // sum over the group; `red` is __shared__ scratch of >= kWarps entries
  __device__ static long long sum(long long x, long long *red) {
    if constexpr (kWarp) {
      return group_sum<GS>(x);
    } else {
      x = warp_sum(x);
      const int w = threadIdx.x >> 5;
      __syncthreads();
      if ((threadIdx.x & 31) == 0) red[w] = x;
      __syncthreads();
      long long t = 0;
#pragma unroll
      for (int i = 0; i < kWarps; ++i) t += red[i];
      return t;
    }
  }

  __device__ static void argmax(long long &g, int32_t &x, long long *rg, int32_t *rx) {
    if constexpr (kWarp) {
      group_argmax<GS>(g, x);
    } else {
      group_argmax<32>(g, x);
      const int w = threadIdx.x >> 5;
      __syncthreads();
      if ((threadIdx.x & 31) == 0) {
        rg[w] = g;
        rx[w] = x;
      }
      __syncthreads();
      g = rg[0];
      x = rx[0];
#pragma unroll
      for (int i = 1; i < kWarps; ++i)
        if (better(rg[i], rx[i], g, x)) {
          g = rg[i];
          x = rx[i];
        }
    }
  }
};

// Calls body(i, active) for every index i of a bin list of `count` entries,
// uniformly over each warp (GS <= 32) or block (GS > 32).
template <int GS, typename Body>
__device__ __forceinline__ void for_each_vertex(int64_t count, Body body) {
  if constexpr (GS <= 32) {
    constexpr int gpw = 32 / GS;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * gpw; base < count; base += nw * gpw) {
      const int64_t i = base + lane / GS;
      body(i, i < count);
    }
  } else {
    for (int64_t i = blockIdx.x; i < count; i += gridDim.x) body(i, true);
  }
}

// Block-wide sums of per-thread counters added once per block to device scalars.
__device__ __forceinline__ void flush_block_sum(long long x, long long *dst) {
  __shared__ long long red[32];
  x = warp_sum(x);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    long long t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
    t = warp_sum(t);
    if (threadIdx.x == 0 && t != 0) atomicAdd((unsigned long long *)dst, (unsigned long long)t);
  }
}

}  // namespace lc
