// lc_scan.cuh — device-wide exclusive prefix sums and stream compaction.
//
// Three launches over tiles of kScanTile inputs: per-tile totals, a scan of
// the tile totals, then a per-tile block scan that hands every input its
// exclusive prefix.  Inputs and outputs are functors, so the flag of a
// compaction and the scatter it feeds are fused into the scan instead of
// materialising an index array.  Used for: label compaction (ids in use),
// new-singleton ids (free ids, empty-cluster movers), coarse CSR offsets and
// the stream compaction of the contraction tables (Algorithm 4's
// ExclusivePrefixSum and StreamCompaction).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lc {

constexpr int kScanThreads = 256;
constexpr int kScanRows = 16;
constexpr int kScanTile = kScanThreads * kScanRows;

inline int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }
// Elements of scratch a scan over n inputs needs (tile totals + grand total).
inline int64_t scan_scratch(int64_t n) { return scan_tiles(n) + 2; }

// Exclusive block scan of one value per thread (blockDim.x == kScanThreads).
template <typename T>
__device__ __forceinline__ T block_exclusive(T x, T *warp_tot, T &total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    constexpr int nw = kScanThreads / 32;
    T t = lane < nw ? warp_tot[lane] : T(0);
    T ti = t;
#pragma unroll
    for (int o = 1; o < nw; o <<= 1) {
      T y = __shfl_up_sync(0xFFFFFFFFu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < nw) warp_tot[lane] = ti - t;
    if (lane == nw - 1) warp_tot[nw] = ti;
  }
  __syncthreads();
  T res = incl - x + warp_tot[wid];
  total = warp_tot[kScanThreads / 32];
  __syncthreads();
  return res;
}

template <typename T, typename In>
__global__ void __launch_bounds__(kScanThreads) k_scan_tile_totals(In in, int64_t n, T *tile_tot,
                                                                   const int *skip) {
  if (skip && *skip == 0) return;
  __shared__ T wt[kScanThreads / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  T s = 0;
#pragma unroll 4
  for (int r = 0; r < kScanRows; ++r) {
    int64_t i = base + r * kScanThreads + threadIdx.x;
    if (i < n) s += in(i);
  }
  T total;
  block_exclusive<T>(s, wt, total);
  if (threadIdx.x == 0) tile_tot[blockIdx.x] = total;
}

// Single block: exclusive scan of tile totals in place; tile_tot[tiles] = grand total.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_tile_prefix(T *tile_tot, int64_t tiles,
                                                                   const int *skip) {
  if (skip && *skip == 0) return;
  __shared__ T wt[kScanThreads / 32 + 1];
  T carry = 0;
  for (int64_t b = 0; b < tiles; b += kScanThreads) {
    int64_t i = b + threadIdx.x;
    T x = i < tiles ? tile_tot[i] : T(0);
    T total;
    T ex = block_exclusive<T>(x, wt, total);
    if (i < tiles) tile_tot[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) tile_tot[tiles] = carry;
}

// out(i, prefix, value) is called for every i < n with the exclusive prefix.
template <typename T, typename In, typename Out>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(In in, Out out, int64_t n,
                                                             const T *tile_tot, const int *skip) {
  if (skip && *skip == 0) return;
  __shared__ T wt[kScanThreads / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  T carry = tile_tot[blockIdx.x];
  for (int r = 0; r < kScanRows; ++r) {
    int64_t i = base + r * kScanThreads + threadIdx.x;
    T x = i < n ? in(i) : T(0);
    T total;
    T ex = block_exclusive<T>(x, wt, total);
    if (i < n) out(i, carry + ex, x);
    carry += total;
  }
}

// Runs the scan.  scratch: scan_scratch(n) elements of T; the grand total is
// left in scratch[scan_tiles(n)].  If `skip` is non-null and *skip == 0 on
// the device when a launch starts, the launch does nothing.
template <typename T, typename In, typename Out>
void scan_apply(int64_t n, In in, Out out, T *scratch, cudaStream_t s, const int *skip = nullptr) {
  const int64_t tiles = scan_tiles(n);
  if (tiles == 0) {
    cudaMemsetAsync(scratch, 0, sizeof(T), s);
    return;
  }
  k_scan_tile_totals<T, In><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, scratch, skip);
  k_scan_tile_prefix<T><<<1, kScanThreads, 0, s>>>(scratch, tiles, skip);
  k_scan_apply<T, In, Out><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, scratch, skip);
}

}  // namespace lc
