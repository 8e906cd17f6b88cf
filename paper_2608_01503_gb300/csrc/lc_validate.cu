// lc_validate.cu — CSR precondition checks and the sums the exactness guards
// need (Section II: positive integer edge weights, undirected graph stored in
// both directions; vertex weights may also be zero, the weighted degree of an
// isolated vertex under modularity).  One warp per vertex streams its row once.
#include "lc_group.cuh"
#include "lc_internal.cuh"
#include "lc_validate.cuh"

namespace lc {

__device__ __forceinline__ void report(GraphStats *st, int code, int64_t v) {
  const unsigned long long key = ((unsigned long long)code << 40) | (unsigned long long)(v & 0xFFFFFFFFFFll);
  atomicMin(&st->err_key, key);
}

// SplitMix64 output mix, used as an edge fingerprint.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void __launch_bounds__(256) k_stats(LevelGraph g, int validate, GraphStats *st) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  long long T = 0, V = 0, sw2 = 0;
  unsigned long long f1 = 0, f2 = 0;
  for (int64_t v = warp; v < g.n; v += nw) {
    const int64_t beg = g.rp[v], end = g.rp[v + 1];
    if (lane == 0) {
      const long long w = g.vw[v];
      V += w;
      sw2 += w * w;
      if (validate && w < 0) report(st, LC_ERR_WEIGHT, v);
    }
    if (end < beg || beg < 0 || end > g.nnz) {
      if (lane == 0) report(st, LC_ERR_ARG, v);
      continue;
    }
    for (int64_t e = beg + lane; e < end; e += 32) {
      const int32_t u = g.col[e];
      const int32_t w = g.ew[e];
      T += w;
      if (validate) {
        if (u < 0 || u >= g.n) {
          report(st, LC_ERR_ARG, v);
          continue;
        }
        if (u == v) report(st, LC_ERR_SELF_LOOP, v);
        if (e > beg && g.col[e - 1] >= u) report(st, LC_ERR_DUPLICATE, v);
        if (w <= 0) report(st, LC_ERR_WEIGHT, v);
        const unsigned long long a = (unsigned long long)(v < u ? v : u);
        const unsigned long long b = (unsigned long long)(v < u ? u : v);
        const unsigned long long key = (a << 32) | b;
        const unsigned long long h1 = mix64(key ^ ((unsigned long long)(uint32_t)w * 0x9E3779B97F4A7C15ull));
        const unsigned long long h2 = mix64((key + 0x632BE59BD9B4E019ull) ^ ((unsigned long long)(uint32_t)w << 17));
        if (v < u) {
          f1 += h1;
          f2 += h2;
        } else {
          f1 -= h1;
          f2 -= h2;
        }
      }
    }
  }
  T = warp_sum(T);
  V = warp_sum(V);
  sw2 = warp_sum(sw2);
  f1 = warp_sum(f1);
  f2 = warp_sum(f2);
  if (lane == 0) {
    atomicAdd((unsigned long long *)&st->T, (unsigned long long)T);
    atomicAdd((unsigned long long *)&st->V, (unsigned long long)V);
    atomicAdd((unsigned long long *)&st->sw2, (unsigned long long)sw2);
    if (f1) atomicAdd(&st->fp1, f1);
    if (f2) atomicAdd(&st->fp2, f2);
  }
}

__global__ void k_labels_in_range(const int32_t *__restrict__ C, int64_t n, int64_t limit,
                                  GraphStats *st) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    if (C[v] < 0 || C[v] >= limit) report(st, LC_ERR_ARG, v);
}

void launch_stats(const LevelGraph &g, int validate, GraphStats *st, cudaStream_t s) {
  int64_t blocks = (g.n * 32 + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_stats<<<(unsigned)blocks, 256, 0, s>>>(g, validate, st);
}

void launch_labels_in_range(const int32_t *C, int64_t n, int64_t limit, GraphStats *st,
                            cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_labels_in_range<<<(unsigned)blocks, 256, 0, s>>>(C, n, limit, st);
}

}  // namespace lc
