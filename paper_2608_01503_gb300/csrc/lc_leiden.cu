// lc_leiden.cu — pLeiden's own steps (Section V): LocalMoveAlt (Section
// V-A), the parallel refinement pLeidenR (Algorithm 6) and Downsample
// (Algorithm 5).  LocalMovePasses and the contraction are the Louvain+
// kernels.
#include <climits>
#include <utility>

#include "lc_group.cuh"
#include "lc_leiden.cuh"
#include "lc_pass.cuh"
#include "lc_scan.cuh"

namespace lc {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

unsigned ld_grid(int64_t n, int per_block) {
  const int64_t b = (n + per_block - 1) / per_block;
  return (unsigned)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

// ------------------------------------------------------- LocalMoveAlt

struct AltIn {
  const int32_t *D;
  const int64_t *delta;
  __device__ int64_t operator()(int64_t v) const { return D[v] != kNone && delta[v] > 0; }
};
struct AltOut {
  int32_t *list;
  __device__ void operator()(int64_t v, int64_t pos, int64_t x) const {
    if (x) list[pos] = (int32_t)v;
  }
};

__global__ void k_sizes(const int32_t *__restrict__ C, int32_t *__restrict__ size, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&size[C[v]], 1);
}

constexpr int kAltThreads = 1024;

// One block applies the listed moves in order.  Per move: the exact gains
// of staying and of the destination under all earlier moves (block sums
// over the row), the running total and the best prefix; a move to the
// empty cluster takes the smallest unused id (a vertex already alone keeps
// its id).  At the end the moves after the best prefix are undone.
__global__ void __launch_bounds__(kAltThreads) k_local_move_alt(LevelGraph g, const GraphParam *gp,
                                                               int32_t *C, const int32_t *D,
                                                               int64_t *W, int32_t *size,
                                                               const int32_t *list, const int64_t *m_ptr,
                                                               int32_t *to, int32_t *old,
                                                               int64_t *scal, int *error) {
  __shared__ long long red_c[kAltThreads / 32], red_d[kAltThreads / 32];
  __shared__ long long s_cum, s_best;
  __shared__ int64_t s_bestk, s_hint;
  __shared__ int32_t s_need, s_found;
  const int64_t m = *m_ptr;
  const GraphParam P = gp[0];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    s_cum = 0;
    s_best = 0;
    s_bestk = 0;
    s_hint = 0;
  }
  __syncthreads();
  for (int64_t k = 0; k < m; ++k) {
    const int32_t v = list[k];
    const int32_t Dv = D[v], Cv = C[v];
    long long sc = 0, sd = 0;
    for (int64_t e = g.rp[v] + threadIdx.x; e < g.rp[v + 1]; e += kAltThreads) {
      const int32_t X = C[g.col[e]];
      const int32_t w = g.ew[e];
      if (X == Cv) sc += w;
      if (Dv >= 0 && X == Dv) sd += w;
    }
    sc = warp_sum(sc);
    sd = warp_sum(sd);
    if (lane == 0) {
      red_c[wid] = sc;
      red_d[wid] = sd;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long Sc = 0, Sd = 0;
      for (int i = 0; i < kAltThreads / 32; ++i) {
        Sc += red_c[i];
        Sd += red_d[i];
      }
      const long long wv = g.vw[v];
      const long long gC = P.Lam * Sc - P.mu * wv * (W[Cv] - wv);
      const long long gD = Dv >= 0 ? P.Lam * Sd - P.mu * wv * W[Dv] : 0;
      s_cum += 2 * (gD - gC);
      if (s_cum > s_best) {
        s_best = s_cum;
        s_bestk = k + 1;
      }
      s_need = Dv == kEmpty && size[Cv] > 1;
      s_found = s_need ? INT_MAX : (Dv == kEmpty ? Cv : Dv);
    }
    __syncthreads();
    if (s_need) {  // block-wide search for the smallest unused id from the hint
      bool done = false;
      for (int64_t base = s_hint; base < g.n && !done; base += kAltThreads) {
        const int64_t x = base + threadIdx.x;
        const bool z = x < g.n && size[x] == 0;
        if (z) atomicMin(&s_found, (int32_t)x);
        done = __syncthreads_or(z);
      }
      if (threadIdx.x == 0 && s_found == INT_MAX) {  // cannot happen: C[v] has >= 2 members
        *error = 1;
        s_found = Cv;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const int32_t t = s_found;
      const long long wv = g.vw[v];
      old[k] = Cv;
      to[k] = t;
      W[Cv] -= wv;
      W[t] += wv;
      size[Cv] -= 1;
      size[t] += 1;
      C[v] = t;
      if (s_need) s_hint = (int64_t)t + 1;
      if (size[Cv] == 0 && Cv < s_hint) s_hint = Cv;
    }
    __syncthreads();
  }
  const int64_t bk = s_bestk;
  for (int64_t k = bk + threadIdx.x; k < m; k += kAltThreads) C[list[k]] = old[k];
  if (threadIdx.x == 0) scal[1] = bk;
}

// ----------------------------------------------------------- pLeidenR

constexpr uint64_t kK = 1ull << 62;  // keys f in [0, K); a fixed singleton takes 2K - f

enum : uint8_t { kInU = 1, kKept = 2, kChild = 4, kFixed = 8 };

__device__ __forceinline__ bool key_less(uint64_t fa, int64_t a, uint64_t fb, int64_t b) {
  return fa < fb || (fa == fb && a < b);
}

// w'(u,v) >= 0 for an edge, Lambda-scaled: Lam w(u,v) - mu w(u) w(v).
__device__ __forceinline__ bool edge_ok(const GraphParam &P, int32_t w, long long wu, long long wv) {
  return P.Lam * (long long)w - P.mu * wu * wv >= 0;
}

// The per-vertex refinement kernels take the level's degree bins: one
// thread per vertex up to degree 32 (GS = 1), one warp above (GS = 32).

template <int GS>
__device__ __forceinline__ long long grp_sum(long long x) {
  if constexpr (GS == 1) return x;
  else return warp_sum(x);
}

// S(v, B[v]), membership of U, and the key f(v).
template <int GS>
__global__ void __launch_bounds__(kThreads) k_ref_self(LevelGraph g, const GraphParam *gp,
                                                       const int32_t *__restrict__ list, int64_t count,
                                                       const int32_t *__restrict__ B,
                                                       const int64_t *__restrict__ WB,
                                                       int64_t *__restrict__ SB, uint8_t *__restrict__ flags,
                                                       uint64_t *__restrict__ f, RefRec *__restrict__ rec,
                                                       uint32_t seed, int32_t level) {
  const GraphParam P = gp[0];
  const int r = Grp<GS>::rank();
  for_each_vertex<GS>(count, [&](int64_t i, bool active) {
    const int32_t v = active ? list[i] : 0;
    const int32_t Bv = active ? B[v] : 0;
    const int64_t beg = active ? g.rp[v] : 0, end = active ? g.rp[v + 1] : 0;
    long long sb = 0;
    for (int64_t e = beg + r; e < end; e += GS)
      if (B[__ldg(g.col + e)] == Bv) sb += __ldg(g.ew + e);
    sb = grp_sum<GS>(sb);
    if (active && r == 0) {
      const long long wv = g.vw[v];
      const bool inU = P.Lam * sb - P.mu * wv * (WB[Bv] - wv) >= 0;
      SB[v] = sb;
      flags[v] = inU ? kInU : 0;
      f[v] = stream_rand(seed, level, 1, v) >> 2;
      rec[v] = RefRec{Bv, inU ? 1 : 0, wv};
    }
  });
}

// ChooseRandom: among v itself and the qualifying neighbours, the
// candidate c with the smallest (rand(v << 32 | c), c) of stream 0 --
// uniform, and independent of the order of the row.
template <int GS>
__global__ void __launch_bounds__(kThreads) k_ref_choose(LevelGraph g, const GraphParam *gp,
                                                         const int32_t *__restrict__ list, int64_t count,
                                                         const RefRec *__restrict__ rec,
                                                         int32_t *__restrict__ H, uint32_t seed,
                                                         int32_t level) {
  const GraphParam P = gp[0];
  const int r = Grp<GS>::rank();
  for_each_vertex<GS>(count, [&](int64_t i, bool active) {
    const int32_t v = active ? list[i] : 0;
    const RefRec rv = active ? rec[v] : RefRec{0, 0, 0};
    const bool inU = active && rv.inU;
    uint64_t best = ~0ull;
    int32_t h = v;
    if (inU) {
      best = stream_rand(seed, level, 0, ((int64_t)v << 32) | v);
      for (int64_t e = g.rp[v] + r; e < g.rp[v + 1]; e += GS) {
        const int32_t u = __ldg(g.col + e);
        const RefRec ru = rec[u];  // one gather: B[u], u in U, w(u)
        if (ru.inU && ru.B == rv.B && edge_ok(P, __ldg(g.ew + e), ru.w, rv.w)) {
          const uint64_t x = stream_rand(seed, level, 0, ((int64_t)v << 32) | u);
          if (x < best || (x == best && u < h)) {
            best = x;
            h = u;
          }
        }
      }
    }
    if constexpr (GS > 1) {
#pragma unroll
      for (int o = GS / 2; o > 0; o >>= 1) {
        const uint64_t ob = __shfl_xor_sync(0xFFFFFFFFu, best, o);
        const int32_t oh = __shfl_xor_sync(0xFFFFFFFFu, h, o);
        if (ob < best || (ob == best && oh < h)) {
          best = ob;
          h = oh;
        }
      }
    }
    if (active && r == 0) H[v] = inU ? h : v;
  });
}

__global__ void k_ref_keep(const int32_t *__restrict__ H, const uint64_t *__restrict__ f,
                           uint8_t *__restrict__ flags, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t h = H[v];
    if (h != v && key_less(f[h], h, f[v], v)) {  // flags bytes are updated with word atomics
      atomicOr(reinterpret_cast<unsigned int *>(flags + (v & ~3ll)), (unsigned)kKept << (8 * (v & 3)));
      atomicOr(reinterpret_cast<unsigned int *>(flags + (h & ~3)), (unsigned)kChild << (8 * (h & 3)));
    }
  }
}

// A vertex whose edge was dropped and that no kept edge reaches takes the
// key 2K - f.
__global__ void k_ref_fix(const int32_t *__restrict__ H, uint64_t *__restrict__ f,
                          uint8_t *__restrict__ flags, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t fl = flags[v];
    if (H[v] != v && !(fl & (kKept | kChild))) {
      f[v] = 2 * kK - f[v];
      flags[v] = fl | kFixed;
    }
  }
}

// The fixed vertices test their edge again against the final keys; then
// every vertex points at its parent (or itself).
__global__ void k_ref_parent(const int32_t *__restrict__ H, const uint64_t *__restrict__ f,
                             const uint8_t *__restrict__ flags, int32_t *__restrict__ root, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t fl = flags[v];
    const int32_t h = H[v];
    bool kept = fl & kKept;
    if (fl & kFixed) kept = key_less(f[h], h, f[v], v);
    root[v] = kept ? h : (int32_t)v;
  }
}

// Roots by following parents (keys strictly decrease towards the root, so
// there are no cycles; with random keys a tree has logarithmic expected
// depth).  parent and root are separate arrays; a walk longer than n sets
// the error flag.
__global__ void k_ref_roots(const int32_t *__restrict__ parent, int32_t *__restrict__ root, int64_t n,
                            int *error) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = (int32_t)v;
    int64_t steps = 0;
    for (int32_t p = parent[r]; p != r && steps <= n; p = parent[r]) {
      r = p;
      ++steps;
    }
    if (steps > n) *error = 1;
    root[v] = r;
  }
}

// Checks that every root is final and packs (root, key) per vertex.
__global__ void k_ref_check_roots(const int32_t *__restrict__ root, const uint64_t *__restrict__ f,
                                  KeyRec *__restrict__ krec, int64_t n, int *error) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = root[v];
    if (root[r] != r) *error = 1;
    krec[v] = KeyRec{r, 0, f[v]};
  }
}

// Weight to the earlier vertices of the tree (same root, smaller key) and
// the vertex's term of w(C, B minus C) along the tree order.
template <int GS>
__global__ void __launch_bounds__(kThreads) k_ref_sv(LevelGraph g, const int32_t *__restrict__ list,
                                                     int64_t count, const KeyRec *__restrict__ krec,
                                                     const int64_t *__restrict__ SB,
                                                     int64_t *__restrict__ Sv, int64_t *__restrict__ tv) {
  const int r = Grp<GS>::rank();
  for_each_vertex<GS>(count, [&](int64_t i, bool active) {
    const int32_t v = active ? list[i] : 0;
    const KeyRec kv = active ? krec[v] : KeyRec{0, 0, 0};
    const int64_t beg = active ? g.rp[v] : 0, end = active ? g.rp[v + 1] : 0;
    long long s = 0;
    for (int64_t e = beg + r; e < end; e += GS) {
      const int32_t u = __ldg(g.col + e);
      const KeyRec ku = krec[u];  // one gather: root and key of u
      if (ku.root == kv.root && key_less(ku.f, u, kv.f, v)) s += __ldg(g.ew + e);
    }
    s = grp_sum<GS>(s);
    if (active && r == 0) {
      Sv[v] = s;
      tv[v] = SB[v] - 2 * s;
    }
  });
}

// ------------------------------------------- LSD radix sort (8-bit digits)

constexpr int kRadixRows = 16;
constexpr int kRadixTile = kThreads * kRadixRows;

__global__ void __launch_bounds__(kThreads) k_radix_hist(const uint64_t *__restrict__ key, int64_t n,
                                                         int shift, int32_t *__restrict__ hist,
                                                         int64_t tiles) {
  __shared__ int32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  for (int r = 0; r < kRadixRows; ++r) {
    const int64_t i = base + r * kThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(key[i] >> shift) & 255], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = cnt[threadIdx.x];
}

struct HistIn {
  const int32_t *h;
  __device__ int64_t operator()(int64_t i) const { return h[i]; }
};
struct HistOut {
  int32_t *h;
  __device__ void operator()(int64_t i, int64_t pos, int64_t) const { h[i] = (int32_t)pos; }
};

// Stable scatter: elements are taken in input order, 256 per round; equal
// digits within a warp are ranked with __match_any_sync, across warps with
// per-warp counts, across rounds with running bucket offsets.
__global__ void __launch_bounds__(kThreads) k_radix_scatter(const uint64_t *__restrict__ kin,
                                                            const int32_t *__restrict__ vin,
                                                            uint64_t *__restrict__ kout,
                                                            int32_t *__restrict__ vout, int64_t n,
                                                            int shift, const int32_t *__restrict__ off,
                                                            int64_t tiles) {
  __shared__ int32_t bucket[256];
  __shared__ int32_t wcnt[kWarps][256];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  bucket[threadIdx.x] = off[(int64_t)threadIdx.x * tiles + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  for (int r = 0; r < kRadixRows; ++r) {
    for (int w = 0; w < kWarps; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = base + r * kThreads + threadIdx.x;
    const bool live = i < n;
    uint64_t k = 0;
    int32_t val = 0;
    int d = 256 + lane;  // distinct dummy digits for lanes past the end
    if (live) {
      k = kin[i];
      val = vin[i];
      d = (int)((k >> shift) & 255);
    }
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (live && rank == 0) wcnt[wid][d] = __popc(peers);
    __syncthreads();
    if (live) {
      int at = bucket[d] + rank;
      for (int w = 0; w < wid; ++w) at += wcnt[w][d];
      kout[at] = k;
      vout[at] = val;
    }
    __syncthreads();
    int add = 0;
    for (int w = 0; w < kWarps; ++w) add += wcnt[w][threadIdx.x];
    bucket[threadIdx.x] += add;
  }
}

// Sorts (key, val) pairs by key, stably, over the low `bits` bits; the
// result is left in (k0, v0).
void radix_sort(uint64_t *k0, int32_t *v0, uint64_t *k1, int32_t *v1, int64_t n, int bits,
                int32_t *hist, int64_t *scan64, cudaStream_t s) {
  const int64_t tiles = (n + kRadixTile - 1) / kRadixTile;
  if (tiles == 0) return;
  for (int shift = 0; shift < bits; shift += 8) {
    k_radix_hist<<<(unsigned)tiles, kThreads, 0, s>>>(k0, n, shift, hist, tiles);
    scan_apply<int64_t>(256 * tiles, HistIn{hist}, HistOut{hist}, scan64, s);
    k_radix_scatter<<<(unsigned)tiles, kThreads, 0, s>>>(k0, v0, k1, v1, n, shift, hist, tiles);
    std::swap(k0, k1);
    std::swap(v0, v1);
  }
  if ((bits + 7) / 8 % 2 == 1) {  // odd number of passes: the result is in (k1, v1) of the caller
    cudaMemcpyAsync(k1, k0, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(v1, v0, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
  }
}

// Vertices of trees with more than one vertex (every other vertex stays a
// singleton and takes no part in the sort).
__global__ void k_mark_trees(const int32_t *__restrict__ root, int32_t *__restrict__ mark, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = root[v];
    if (r != v) {
      mark[v] = 1;
      mark[r] = 1;
    }
  }
}
struct MarkIn {
  const int32_t *mark;
  __device__ int64_t operator()(int64_t v) const { return mark[v] != 0; }
};
struct MarkOut {
  int32_t *list;
  __device__ void operator()(int64_t v, int64_t pos, int64_t x) const {
    if (x) list[pos] = (int32_t)v;
  }
};

__global__ void k_tree_sort_keys(const int32_t *__restrict__ list, const uint64_t *__restrict__ f,
                                 uint64_t *__restrict__ key, const int64_t *m_ptr) {
  const int64_t m = *m_ptr;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    key[i] = f[list[i]];
}

// After the sort by (f, id): key = root * m + rank of (f, id).
__global__ void k_tree_keys(const int32_t *__restrict__ order, const int32_t *__restrict__ root,
                            uint64_t *__restrict__ key, int32_t *__restrict__ val, int64_t m) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = order[i];
    key[i] = (uint64_t)root[v] * (uint64_t)m + (uint64_t)i;
    val[i] = v;
  }
}

__global__ void k_positions(const int32_t *__restrict__ order, int64_t *__restrict__ pos,
                            int32_t *__restrict__ first_bad, int64_t m) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    pos[order[i]] = i;
    first_bad[order[i]] = INT_MAX;  // read only at roots
  }
}

struct OrderIn {
  const int32_t *order;
  const int64_t *a;
  __device__ int64_t operator()(int64_t i) const { return a[order[i]]; }
};
struct PosOut {
  int64_t *o;
  __device__ void operator()(int64_t i, int64_t pos, int64_t) const { o[i] = pos; }
};

// Per position of the tree order: the join test of Lemma 1 for the vertex
// joining the cluster of the earlier vertices of its tree; the first
// failing position of each tree is kept.
__global__ void k_ref_test(const int32_t *__restrict__ order, const int32_t *__restrict__ root,
                           const int64_t *__restrict__ pos, const int64_t *__restrict__ ps_w,
                           const int64_t *__restrict__ ps_t, const int64_t *__restrict__ Sv,
                           const int64_t *__restrict__ vw, const int32_t *__restrict__ B,
                           const int64_t *__restrict__ WB, const GraphParam *gp,
                           int32_t *__restrict__ first_bad, int64_t n) {
  const GraphParam P = gp[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = order[i], r = root[v];
    const int64_t i0 = pos[r];
    if (i == i0) continue;
    const long long Wc = ps_w[i] - ps_w[i0], Ec = ps_t[i] - ps_t[i0];
    const bool c1 = P.Lam * Sv[v] - P.mu * vw[v] * Wc >= 0;
    const bool c2 = P.Lam * Ec - P.mu * Wc * (WB[B[v]] - Wc) >= 0;
    if (!(c1 && c2)) atomicMin(&first_bad[r], (int32_t)i);
  }
}

__global__ void k_ref_label(const int32_t *__restrict__ root, const int32_t *__restrict__ mark,
                            const int64_t *__restrict__ pos, const int32_t *__restrict__ first_bad,
                            int32_t *__restrict__ R, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = root[v];
    R[v] = (mark[v] && pos[v] < first_bad[r]) ? r : (int32_t)v;
  }
}

__global__ void k_downsample(const int32_t *__restrict__ Cd, const int32_t *__restrict__ C,
                             int32_t *__restrict__ Cc, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    if (Cd[v] >= 0) Cc[Cd[v]] = C[v];
}

}  // namespace

void launch_local_move_alt(const LevelGraph &g, const GraphParam *gp, int32_t *C, const int32_t *D,
                           const int64_t *delta, int64_t *W, LeidenScratch &ls, int *error,
                           cudaStream_t s) {
  if (g.n == 0) return;
  scan_apply<int64_t>(g.n, AltIn{D, delta}, AltOut{ls.list}, ls.scan64, s);
  cudaMemsetAsync(ls.size, 0, sizeof(int32_t) * (size_t)g.n, s);
  k_sizes<<<ld_grid(g.n, 256), 256, 0, s>>>(C, ls.size, g.n);
  k_local_move_alt<<<1, kAltThreads, 0, s>>>(g, gp, C, D, W, ls.size, ls.list,
                                              ls.scan64 + scan_tiles(g.n), ls.to, ls.list2, ls.scal,
                                              error);
}

int64_t radix_hist_len(int64_t n) { return 256 * ((n + kRadixTile - 1) / kRadixTile) + 256; }

void launch_pleiden_refine(const LevelGraph &g, const Bins &bins, const GraphParam *gp, const int32_t *B,
                           uint32_t seed, int32_t level, int32_t *R, LeidenScratch &ls, int *error,
                           cudaStream_t s) {
  const int64_t n = g.n;
  if (n == 0) return;
  const unsigned gt = ld_grid(n, 256);
  const BinRange lo = bin_range(bins, 0, 2), hi = bin_range(bins, 3, kBins - 1);
  const unsigned glo = ld_grid(lo.count, 256), ghi = ld_grid(hi.count, kWarps);
  if (lo.count) k_ref_self<1><<<glo, kThreads, 0, s>>>(g, gp, lo.list, lo.count, B, ls.WB, ls.SB, ls.flags, ls.f, ls.rec, seed, level);
  if (hi.count) k_ref_self<32><<<ghi, kThreads, 0, s>>>(g, gp, hi.list, hi.count, B, ls.WB, ls.SB, ls.flags, ls.f, ls.rec, seed, level);
  if (lo.count) k_ref_choose<1><<<glo, kThreads, 0, s>>>(g, gp, lo.list, lo.count, ls.rec, ls.H, seed, level);
  if (hi.count) k_ref_choose<32><<<ghi, kThreads, 0, s>>>(g, gp, hi.list, hi.count, ls.rec, ls.H, seed, level);
  k_ref_keep<<<gt, 256, 0, s>>>(ls.H, ls.f, ls.flags, n);
  k_ref_fix<<<gt, 256, 0, s>>>(ls.H, ls.f, ls.flags, n);
  k_ref_parent<<<gt, 256, 0, s>>>(ls.H, ls.f, ls.flags, ls.first_bad, n);  // parents
  k_ref_roots<<<gt, 256, 0, s>>>(ls.first_bad, ls.root, n, error);
  k_ref_check_roots<<<gt, 256, 0, s>>>(ls.root, ls.f, ls.krec, n, error);
  if (lo.count) k_ref_sv<1><<<glo, kThreads, 0, s>>>(g, lo.list, lo.count, ls.krec, ls.SB, ls.Sv, ls.tv);
  if (hi.count) k_ref_sv<32><<<ghi, kThreads, 0, s>>>(g, hi.list, hi.count, ls.krec, ls.SB, ls.Sv, ls.tv);
  // the vertices of multi-vertex trees, ordered by (f, id) and then by
  // (root, rank): trees contiguous, keys ascending within each tree
  cudaMemsetAsync(ls.size, 0, sizeof(int32_t) * (size_t)n, s);
  k_mark_trees<<<gt, 256, 0, s>>>(ls.root, ls.size, n);
  scan_apply<int64_t>(n, MarkIn{ls.size}, MarkOut{ls.list}, ls.scan64, s);
  int64_t m = 0;
  cudaMemcpyAsync(&m, ls.scan64 + scan_tiles(n), sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (m > 0) {
    const unsigned gm = ld_grid(m, 256);
    k_tree_sort_keys<<<gm, 256, 0, s>>>(ls.list, ls.f, ls.key, ls.scan64 + scan_tiles(n));
    radix_sort(ls.key, ls.list, ls.key2, ls.list2, m, 64, ls.hist, ls.scan64, s);
    k_tree_keys<<<gm, 256, 0, s>>>(ls.list, ls.root, ls.key2, ls.list2, m);
    int bits = 1;
    while (bits < 64 && (((unsigned __int128)1) << bits) < (unsigned __int128)n * (unsigned __int128)m) ++bits;
    radix_sort(ls.key2, ls.list2, ls.key, ls.list, m, bits, ls.hist, ls.scan64, s);
    const int32_t *order = ls.list2;
    k_positions<<<gm, 256, 0, s>>>(order, ls.pos, ls.first_bad, m);
    scan_apply<int64_t>(m, OrderIn{order, g.vw}, PosOut{ls.ps_w}, ls.scan64, s);
    scan_apply<int64_t>(m, OrderIn{order, ls.tv}, PosOut{ls.ps_t}, ls.scan64, s);
    k_ref_test<<<gm, 256, 0, s>>>(order, ls.root, ls.pos, ls.ps_w, ls.ps_t, ls.Sv, g.vw, B, ls.WB, gp,
                                  ls.first_bad, m);
  }
  k_ref_label<<<gt, 256, 0, s>>>(ls.root, ls.size, ls.pos, ls.first_bad, R, n);
}

void launch_downsample(const int32_t *Cd, const int32_t *C, int32_t *Cc, int64_t n, cudaStream_t s) {
  if (n > 0) k_downsample<<<ld_grid(n, 256), 256, 0, s>>>(Cd, C, Cc, n);
}

}  // namespace lc
