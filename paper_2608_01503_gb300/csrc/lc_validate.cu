// lc_validate.cu — CSR precondition checks and the sums the exactness guards
// need (Section II: positive integer edge weights, undirected graph stored in
// both directions; vertex weights may also be zero, the weighted degree of an
// isolated vertex under modularity).  The edge checks are load-balanced over
// entries, so a single long row does not serialise them.
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

// acc[g] += x from every lane (warp-uniform call; g < 0 adds nothing).  When
// all contributing lanes share a graph, as almost always, one atomic per warp.
__device__ __forceinline__ void graph_add(long long *acc, int g, long long x) {
  const bool on = g >= 0 && x != 0;
  const unsigned act = __ballot_sync(0xFFFFFFFFu, on);
  if (!act) return;
  const int leader = __ffs(act) - 1;
  const int g0 = __shfl_sync(0xFFFFFFFFu, g, leader);
  if (__all_sync(0xFFFFFFFFu, !on || g == g0)) {
    const long long t = warp_sum(on ? x : 0ll);
    if ((int)(threadIdx.x & 31) == leader) atomicAdd((unsigned long long *)(acc + g0), (unsigned long long)t);
  } else if (on) {
    atomicAdd((unsigned long long *)(acc + g), (unsigned long long)x);
  }
}

// Per-vertex part: vertex-weight sums and checks, row-pointer sanity.
__global__ void __launch_bounds__(256) k_stats_vertices(LevelGraph g, int validate, GraphStats *st,
                                                        const int32_t *gid, long long *Vg,
                                                        long long *sw2g) {
  long long V = 0, sw2 = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < g.n;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = base + threadIdx.x;
    long long w = 0;
    if (v < g.n) {
      w = g.vw[v];
      V += w;
      sw2 += w * w;
      if (validate && w < 0) report(st, LC_ERR_WEIGHT, v);
      const int64_t beg = g.rp[v], end = g.rp[v + 1];
      if (end < beg || beg < 0 || end > g.nnz) report(st, LC_ERR_ARG, v);
    }
    if (gid) {
      const int gg = v < g.n ? gid[v] : -1;
      graph_add(Vg, gg, w);
      graph_add(sw2g, gg, w * w);
    }
  }
  V = warp_sum(V);
  sw2 = warp_sum(sw2);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd((unsigned long long *)&st->V, (unsigned long long)V);
    atomicAdd((unsigned long long *)&st->sw2, (unsigned long long)sw2);
  }
}

// Per-edge part, load-balanced: each thread takes kStatsChunk consecutive
// entries, finds the row of the first by binary search on row_ptr and walks
// on.  A warp first copies its tile of 32 x kStatsChunk entries from col and
// ew into shared memory with coalesced loads, transposed (row stride 33) so
// that each thread then reads its own consecutive entries without bank
// conflicts; reading them straight from global memory would touch 32 lines
// per warp load.  Every index stays in range even for a malformed row_ptr
// (that case is reported by the vertex part).
constexpr int kStatsChunk = 32;
constexpr int kStatsTile = 32 * kStatsChunk;  // entries per warp tile
constexpr int kStatsThreads = 128;

__global__ void __launch_bounds__(kStatsThreads) k_stats_edges(LevelGraph g, int validate, GraphStats *st,
                                                               const int32_t *gid, long long *Tg) {
  __shared__ int32_t s_col[kStatsThreads / 32][32 * 33];
  __shared__ int32_t s_ew[kStatsThreads / 32][32 * 33];
  const int lane = threadIdx.x & 31;
  int32_t *tc = s_col[threadIdx.x >> 5];
  int32_t *tw = s_ew[threadIdx.x >> 5];
  const int64_t tiles = (g.nnz + kStatsTile - 1) / kStatsTile;
  const int64_t nwarps = (int64_t)gridDim.x * (kStatsThreads / 32);
  long long T = 0;
  unsigned long long f1 = 0, f2 = 0;
  // warp-uniform loop over tiles
  for (int64_t tile = (int64_t)blockIdx.x * (kStatsThreads / 32) + (threadIdx.x >> 5); tile < tiles;
       tile += nwarps) {
    const int64_t tb = tile * kStatsTile;
    __syncwarp();  // the last tile's reads are done
#pragma unroll 4
    for (int j = 0; j < 32; ++j) {
      const int64_t e = tb + j * 32 + lane;
      if (e < g.nnz) {
        tc[j * 33 + lane] = g.col[e];
        tw[j * 33 + lane] = g.ew[e];
      }
    }
    __syncwarp();
    int cur_g = -1;      // graph of the edges summed into tg so far
    long long tg = 0;
    const int64_t e0 = tb + (int64_t)lane * kStatsChunk;
    if (e0 < g.nnz) {
      const int64_t e1 = e0 + kStatsChunk < g.nnz ? e0 + kStatsChunk : g.nnz;
      int64_t lo = 0, hi = g.n;
      while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (g.rp[mid] <= e0)
          lo = mid;
        else
          hi = mid;
      }
      int64_t v = lo, vbeg = g.rp[v], vend = g.rp[v + 1];
      for (int64_t e = e0; e < e1; ++e) {
        while (e >= vend && v + 1 < g.n) {
          ++v;
          vbeg = vend;
          vend = g.rp[v + 1];
        }
        const int j = (int)(e - e0);
        const int32_t u = tc[lane * 33 + j];
        const int32_t w = tw[lane * 33 + j];
        T += w;
        if (gid) {
          const int gv = gid[v];
          if (gv != cur_g && cur_g >= 0) {  // chunk crosses into the next graph
            atomicAdd((unsigned long long *)&Tg[cur_g], (unsigned long long)tg);
            tg = 0;
          }
          cur_g = gv;
          tg += w;
          if (validate && u >= 0 && u < g.n && gid[u] != gv) report(st, LC_ERR_ARG, v);
        }
        if (!validate) continue;
        if (u < 0 || u >= g.n) {
          report(st, LC_ERR_ARG, v);
          continue;
        }
        if (u == v) report(st, LC_ERR_SELF_LOOP, v);
        if (e > vbeg) {
          // the entry before e: this thread's, the previous thread's last
          // one, or (first thread of the tile) global memory
          const int32_t prev = j > 0 ? tc[lane * 33 + j - 1] : lane > 0 ? tc[(lane - 1) * 33 + 31] : g.col[e - 1];
          if (prev >= u) report(st, LC_ERR_DUPLICATE, v);
        }
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
    if (gid) graph_add(Tg, cur_g, tg);
  }
  T = warp_sum(T);
  f1 = warp_sum(f1);
  f2 = warp_sum(f2);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd((unsigned long long *)&st->T, (unsigned long long)T);
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

void launch_stats(const LevelGraph &g, int validate, GraphStats *st, const int32_t *gid, long long *Tg,
                  long long *Vg, long long *sw2g, cudaStream_t s) {
  auto blocks = [](int64_t items) {
    int64_t b = (items + 255) / 256;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
  };
  k_stats_vertices<<<blocks(g.n), 256, 0, s>>>(g, validate, st, gid, Vg, sw2g);
  if (g.nnz > 0) {
    const int64_t tiles = (g.nnz + kStatsTile - 1) / kStatsTile;
    int64_t b = (tiles + kStatsThreads / 32 - 1) / (kStatsThreads / 32);
    if (b > 152 * 6) b = 152 * 6;  // six blocks per SM (34 KB of shared memory each)
    k_stats_edges<<<(unsigned)b, kStatsThreads, 0, s>>>(g, validate, st, gid, Tg);
  }
}

void launch_labels_in_range(const int32_t *C, int64_t n, int64_t limit, GraphStats *st,
                            cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_labels_in_range<<<(unsigned)blocks, 256, 0, s>>>(C, n, limit, st);
}

}  // namespace lc
