// lc_pass.cu — kernels of one synchronous local-move pass (Algorithm 2 with
// the afterburner filter of Algorithm 3) and the per-level objective.
//
// Every vertex is handled by a group of threads sized to its degree bin (see
// kBinMaxDeg): 8 or 32 lanes holding one neighbour each, a warp, or a block.
// All sums are integer (commutative atomics and shuffles), argmax ties go to
// the smallest cluster id, and the afterburner order is a total order, so
// results do not depend on scheduling.
#include <climits>

#include "lc_group.cuh"
#include "lc_internal.cuh"
#include "lc_pass.cuh"
#include "lc_scan.cuh"

namespace lc {

// ---------------------------------------------------- vertex decision

// Algorithm 2 for one vertex once S(v, C[v]) and the best other cluster
// (gbest, best) are known: the empty-cluster rule, the candidate test with
// temperature phi = phi_n / phi_d, and the afterburner priority.
__device__ __forceinline__ void decide(const PassArgs &a, int32_t v, long long gC, int32_t best,
                                       long long gbest, long long &cntL) {
  if (gC < 0 && (best == kNone || gbest < 0)) {
    best = kEmpty;
    gbest = 0;
  }
  const bool inL = best != kNone &&
                   (__int128)a.phi_d * gbest >= (__int128)(a.phi_d - a.phi_n) * (__int128)gC;
  if (inL) {
    const long long d = gbest - gC;
    a.D[v] = best;
    a.delta[v] = d;
    a.q[v] = eps_bucket(a.m, d);
    cntL++;
  } else {
    a.D[v] = kNone;
  }
}

// ------------------------------------------- first pass (Section IV-A-3)

// Singleton start: the adjacent clusters of v are its neighbours, so the
// gains are read straight from the CSR: g(v,{u}) = Lam*w(u,v) - mu*w(v)*w(u),
// and g(v, C[v]) = 0.
template <int GS>
__global__ void __launch_bounds__(GS > 32 ? GS : 256)
    k_first_pass(PassArgs a, const int32_t *__restrict__ list, int64_t count) {
  __shared__ long long rg[GS > 32 ? GS / 32 : 1];
  __shared__ int32_t rx[GS > 32 ? GS / 32 : 1];
  long long cntL = 0;
  const int r = Grp<GS>::rank();
  for_each_vertex<GS>(count, [&](int64_t i, bool active) {
    const int32_t v = active ? list[i] : 0;
    const int64_t beg = active ? a.g.rp[v] : 0, end = active ? a.g.rp[v + 1] : 0;
    const long long wv = active ? a.g.vw[v] : 0;
    long long gb = LLONG_MIN;
    int32_t xb = kNone;
    for (int64_t e = beg + r; e < end; e += GS) {
      const int32_t u = __ldg(a.g.col + e);
      const long long g = a.m.Lam * (long long)__ldg(a.g.ew + e) - a.m.mu * wv * __ldg(a.g.vw + u);
      if (better(g, u, gb, xb)) {
        gb = g;
        xb = u;
      }
    }
    Grp<GS>::argmax(gb, xb, rg, rx);
    if (active && r == 0) decide(a, v, 0, xb, gb, cntL);
  });
  flush_block_sum(cntL, &a.sc->count_L);
}

// --------------------------------------- aggregation + argmax, bins 0-1

// Each lane holds one neighbour; lanes of a group with the same neighbour
// cluster are matched with __match_any_sync and their weights summed in a
// per-lane shared slot of the lowest matching lane.  S(v, C[v]) is a group
// reduction (the dedicated current-cluster slot of Section IV-A-3).
template <int G>
__global__ void __launch_bounds__(256) k_move_small(PassArgs a, const int32_t *__restrict__ list,
                                                    int64_t count) {
  __shared__ int32_t acc[256];
  long long cntL = 0, phi = 0;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (G - 1);
  const int wbase = threadIdx.x & ~31;
  for_each_vertex<G>(count, [&](int64_t i, bool active) {
    const int32_t v = active ? list[i] : 0;
    const int64_t beg = active ? a.g.rp[v] : 0, deg = active ? a.g.rp[v + 1] - beg : 0;
    const int32_t Cv = active ? a.C[v] : 0;
    const bool has = sub < deg;
    int32_t X = -1, w = 0;
    if (has) {
      const int32_t u = __ldg(a.g.col + beg + sub);
      w = __ldg(a.g.ew + beg + sub);
      X = a.C[u];
    }
    const bool self = has && X == Cv;
    const bool other = has && !self;
    const long long S_self = group_sum<G>((long long)(self ? w : 0));
    const unsigned long long key =
        other ? (((unsigned long long)(lane / G) << 32) | (uint32_t)X) : (0xFFFFFFFF00000000ull | lane);
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
    const int leader = __ffs(peers) - 1;
    acc[threadIdx.x] = 0;
    __syncwarp();
    if (other) atomicAdd(&acc[wbase + leader], w);
    __syncwarp();
    long long wv = 0;
    if (active) wv = a.g.vw[v];
    long long g = LLONG_MIN;
    int32_t x = kNone;
    if (other && lane == leader) {
      g = gain_other(a.m, acc[threadIdx.x], wv, a.W[X]);
      x = X;
    }
    group_argmax<G>(g, x);
    if (active && sub == 0) {
      const long long gC = gain_self(a.m, S_self, wv, a.W[Cv]);
      phi += gC;
      if (a.decide) decide(a, v, gC, x, g, cntL);
    }
    __syncwarp();
  });
  flush_block_sum(cntL, &a.sc->count_L);
  flush_block_sum(phi, &a.sc->phi_acc);
}

// ------------------------------------------ aggregation + argmax, bin 2

// One warp per vertex; a per-warp shared table of cap = pow2 >= 2 deg slots.
__global__ void __launch_bounds__(kBin2Warps * 32)
    k_move_warp(PassArgs a, const int32_t *__restrict__ list, int64_t count) {
  __shared__ unsigned long long tabs[kBin2Warps][kBin2Slots];
  long long cntL = 0, phi = 0;
  const int lane = threadIdx.x & 31;
  unsigned long long *tab = tabs[threadIdx.x >> 5];
  for_each_vertex<32>(count, [&](int64_t i, bool active) {
    if (!active) return;  // warp-uniform: the whole warp shares i
    const int32_t v = list[i];
    const int64_t beg = a.g.rp[v], end = a.g.rp[v + 1];
    const int32_t Cv = a.C[v];
    uint32_t cap = 64;
    while (cap < 2 * (end - beg)) cap <<= 1;
    for (uint32_t s = lane; s < cap; s += 32) tab[s] = kEmptySlot;
    __syncwarp();
    long long self = 0;
    bool ok = true;
    for (int64_t e = beg + lane; e < end; e += 32) {
      const int32_t u = __ldg(a.g.col + e);
      const int32_t w = __ldg(a.g.ew + e);
      const int32_t X = a.C[u];
      if (X == Cv) {
        self += w;
      } else {
        bool fresh = false;
        ok &= table_add(tab, cap, X, w, fresh);
      }
    }
    if (!ok) a.sc->error = 1;
    __syncwarp();
    const long long wv = a.g.vw[v];
    long long gb = LLONG_MIN;
    int32_t xb = kNone;
    for (uint32_t s = lane; s < cap; s += 32) {
      const unsigned long long t = tab[s];
      if (t != kEmptySlot) {
        const int32_t X = slot_key(t);
        const long long g = gain_other(a.m, slot_val(t), wv, a.W[X]);
        if (better(g, X, gb, xb)) {
          gb = g;
          xb = X;
        }
      }
    }
    group_argmax<32>(gb, xb);
    self = warp_sum(self);
    if (lane == 0) {
      const long long gC = gain_self(a.m, self, wv, a.W[Cv]);
      phi += gC;
      if (a.decide) decide(a, v, gC, xb, gb, cntL);
    }
    __syncwarp();
  });
  flush_block_sum(cntL, &a.sc->count_L);
  flush_block_sum(phi, &a.sc->phi_acc);
}

// --------------------------------------- aggregation + argmax, bins 3-4

// One block per vertex.  kShared: table in dynamic shared memory (cap = pow2
// >= 2 deg <= kBin3Slots).  Otherwise the table is the vertex's region
// [2 rp[v], 2 rp[v+1]) of the global scratch, which is clean on entry and
// reset to empty while it is read.
template <int GS, bool kShared>
__global__ void __launch_bounds__(GS) k_move_block(PassArgs a, const int32_t *__restrict__ list,
                                                   int64_t count) {
  extern __shared__ unsigned long long dyn[];
  __shared__ long long rs[GS / 32];
  __shared__ long long rg[GS / 32];
  __shared__ int32_t rx[GS / 32];
  long long cntL = 0, phi = 0;
  for_each_vertex<GS>(count, [&](int64_t i, bool) {
    const int32_t v = list[i];
    const int64_t beg = a.g.rp[v], end = a.g.rp[v + 1];
    const int32_t Cv = a.C[v];
    unsigned long long *tab;
    uint32_t cap;
    if constexpr (kShared) {
      cap = 64;
      while (cap < 2 * (end - beg)) cap <<= 1;
      tab = dyn;
      for (uint32_t s = threadIdx.x; s < cap; s += GS) tab[s] = kEmptySlot;
      __syncthreads();
    } else {
      cap = (uint32_t)(2 * (end - beg));
      tab = a.gtab + 2 * beg;
    }
    long long self = 0;
    bool ok = true;
    for (int64_t e = beg + threadIdx.x; e < end; e += GS) {
      const int32_t u = __ldg(a.g.col + e);
      const int32_t w = __ldg(a.g.ew + e);
      const int32_t X = a.C[u];
      if (X == Cv) {
        self += w;
      } else {
        bool fresh = false;
        ok &= table_add(tab, cap, X, w, fresh);
      }
    }
    if (!ok) a.sc->error = 1;
    __syncthreads();
    const long long wv = a.g.vw[v];
    long long gb = LLONG_MIN;
    int32_t xb = kNone;
    for (uint32_t s = threadIdx.x; s < cap; s += GS) {
      const unsigned long long t = tab[s];
      if (t != kEmptySlot) {
        if constexpr (!kShared) tab[s] = kEmptySlot;
        const int32_t X = slot_key(t);
        const long long g = gain_other(a.m, slot_val(t), wv, a.W[X]);
        if (better(g, X, gb, xb)) {
          gb = g;
          xb = X;
        }
      }
    }
    Grp<GS>::argmax(gb, xb, rg, rx);
    self = Grp<GS>::sum(self, rs);
    if (threadIdx.x == 0) {
      const long long gC = gain_self(a.m, self, wv, a.W[Cv]);
      phi += gC;
      if (a.decide) decide(a, v, gC, xb, gb, cntL);
    }
    __syncthreads();
  });
  flush_block_sum(cntL, &a.sc->count_L);
  flush_block_sum(phi, &a.sc->phi_acc);
}

// ------------------------------------------------ afterburner (Algorithm 3)

// For each candidate v: delta_v adjusted by every adjacent candidate u that
// precedes v in the order, by the exact change of v's two gains when u moves
// from C[u] to D[u]; v survives iff the adjusted delta is >= 0.
template <int GS>
__global__ void __launch_bounds__(GS > 32 ? GS : 256)
    k_afterburner(PassArgs a, const int32_t *__restrict__ list, int64_t count) {
  __shared__ long long rs[GS > 32 ? GS / 32 : 1];
  long long cntM = 0;
  const int r = Grp<GS>::rank();
  for_each_vertex<GS>(count, [&](int64_t i, bool active) {
    const int32_t v = active ? list[i] : 0;
    const int32_t Dv = active ? a.D[v] : kNone;
    const bool cand = Dv != kNone;
    long long acc = 0;
    if (cand) {
      const int64_t beg = a.g.rp[v], end = a.g.rp[v + 1];
      const int32_t Cv = a.C[v];
      const long long qv = a.q[v], wv = a.g.vw[v];
      const uint32_t hv = fmix32((uint32_t)v ^ a.m.seed);
      for (int64_t e = beg + r; e < end; e += GS) {
        const int32_t u = __ldg(a.g.col + e);
        const int32_t Du = a.D[u];
        if (Du == kNone) continue;
        const long long qu = a.q[u];
        if (!earlier(qu, fmix32((uint32_t)u ^ a.m.seed), u, qv, hv, v)) continue;
        const int32_t Cu = a.C[u];
        const long long aw = a.m.Lam * (long long)__ldg(a.g.ew + e) - a.m.mu * a.g.vw[u] * wv;
        if (Cv == Cu)
          acc += aw;
        else if (Dv == Cu)
          acc -= aw;
        if (Cv == Du)
          acc -= aw;
        else if (Dv >= 0 && Dv == Du)
          acc += aw;
      }
    }
    if constexpr (GS <= 32) {
      acc = group_sum<GS>(acc);
    } else {
      acc = Grp<GS>::sum(acc, rs);
    }
    if (active && r == 0) {
      const bool keep = cand && a.delta[v] + acc >= 0;
      a.M[v] = keep;
      cntM += keep;
    }
  });
  flush_block_sum(cntM, &a.sc->count_M);
}

// ---------------------------------------------------- objective, S_self

// Phi(C) = sum over v of g(v, C[v]) (Eq. 1 regrouped per vertex): sweeps
// each row for neighbours in C[v].
template <int GS>
__global__ void __launch_bounds__(GS > 32 ? GS : 256)
    k_objective(PassArgs a, const int32_t *__restrict__ list, int64_t count) {
  __shared__ long long rs[GS > 32 ? GS / 32 : 1];
  long long phi = 0;
  const int r = Grp<GS>::rank();
  for_each_vertex<GS>(count, [&](int64_t i, bool active) {
    const int32_t v = active ? list[i] : 0;
    long long self = 0;
    int32_t Cv = 0;
    if (active) {
      const int64_t beg = a.g.rp[v], end = a.g.rp[v + 1];
      Cv = a.C[v];
      for (int64_t e = beg + r; e < end; e += GS)
        if (a.C[__ldg(a.g.col + e)] == Cv) self += __ldg(a.g.ew + e);
    }
    if constexpr (GS <= 32) {
      self = group_sum<GS>(self);
    } else {
      self = Grp<GS>::sum(self, rs);
    }
    if (active && r == 0) phi += gain_self(a.m, self, a.g.vw[v], a.W[Cv]);
  });
  flush_block_sum(phi, &a.sc->phi_acc);
}

// ----------------------------------------------------------- update

// Apply D for M (Algorithm 2, Update): real destinations move now; movers
// to a new empty cluster leave their cluster and are flagged for ids.
__global__ void k_apply(PassArgs a, uint8_t *__restrict__ E) {
  long long empties = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.g.n;
       v += (int64_t)gridDim.x * blockDim.x) {
    uint8_t e = 0;
    if (a.M[v]) {
      const int32_t Dv = a.D[v], Cv = a.C[v];
      const long long wv = a.g.vw[v];
      atomicAdd((unsigned long long *)&a.W[Cv], (unsigned long long)(-wv));
      if (Dv >= 0) {
        a.C[v] = Dv;
        atomicAdd((unsigned long long *)&a.W[Dv], (unsigned long long)wv);
      } else {
        e = 1;
        empties++;
      }
    }
    E[v] = e;
  }
  __shared__ long long red[32];
  long long x = warp_sum(empties);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    if (t) atomicAdd(&a.sc->empty_movers, (int)t);
  }
}

// Empty-cluster movers, ascending, take the ascending ids that are unused
// once every other move is applied.  Ids in use are marked from the labels
// (vertex weights may be zero, so W(x) == 0 does not mean x is empty).
__global__ void k_mark_occupied(const int32_t *__restrict__ C, const uint8_t *__restrict__ E,
                                int32_t *__restrict__ used, int64_t n, const int *k) {
  if (*k == 0) return;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    if (!E[v]) used[C[v]] = 1;
}
__global__ void k_zero_if(int32_t *__restrict__ used, int64_t n, const int *k) {
  if (*k == 0) return;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    used[v] = 0;
}
struct FreeFlag {
  const int32_t *used;
  __device__ int32_t operator()(int64_t x) const { return used[x] == 0 ? 1 : 0; }
};
struct FreeEmit {
  int32_t *freelist;
  const int *k;
  __device__ void operator()(int64_t x, int32_t pos, int32_t f) const {
    if (f && pos < *k) freelist[pos] = (int32_t)x;
  }
};
struct MoverFlag {
  const uint8_t *E;
  __device__ int32_t operator()(int64_t v) const { return E[v]; }
};
struct MoverEmit {
  const int32_t *freelist;
  int32_t *C;
  int64_t *W;
  const int64_t *vw;
  int64_t n;
  int *error;
  __device__ void operator()(int64_t v, int32_t pos, int32_t f) const {
    if (f) {
      // there are always at least as many free ids as movers; a list entry
      // outside [0, n) would be a bound violation, reported, never used
      const int32_t x = freelist[pos];
      if (x < 0 || x >= n) {
        *error = 1;
        return;
      }
      C[v] = x;
      W[x] = vw[v];
    }
  }
};

// ----------------------------------------------------------- best-of

__global__ void k_pass_begin(Scalars *sc) {
  sc->count_L = 0;
  sc->count_M = 0;
  sc->empty_movers = 0;
}

// Algorithm 2's best-of test on the objective accumulated in phi_acc.
__global__ void k_bestof_test(Scalars *sc) {
  const long long p = sc->phi_acc;
  if (p > sc->phi_out) {
    sc->phi_out = p;
    sc->improved = 1;
  } else {
    sc->improved = 0;
  }
  sc->phi_acc = 0;
}

__global__ void k_bestof_copy(const Scalars *sc, const int32_t *__restrict__ C,
                              int32_t *__restrict__ C_out, int64_t n) {
  if (!sc->improved) return;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    C_out[v] = C[v];
}

// ------------------------------------------------------------ helpers

__global__ void k_iota(int32_t *C, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    C[v] = (int32_t)v;
}

__global__ void k_cluster_weights(const int32_t *__restrict__ C, const int64_t *__restrict__ vw,
                                  int64_t *W, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    atomicAdd((unsigned long long *)&W[C[v]], (unsigned long long)vw[v]);
}

// ------------------------------------------------------------ binning

struct BinFlag {
  const int64_t *rp;
  int64_t lo, hi;  // lo < deg <= hi
  __device__ int32_t operator()(int64_t v) const {
    const int64_t d = rp[v + 1] - rp[v];
    return (d > lo && d <= hi) ? 1 : 0;
  }
};
struct BinEmit {
  int32_t *lists;
  const int32_t *off;  // start of this bin in lists
  __device__ void operator()(int64_t v, int32_t pos, int32_t f) const {
    if (f) lists[*off + pos] = (int32_t)v;
  }
};

__global__ void k_bin_next_offset(int32_t *offs, int k, const int32_t *total) {
  offs[k + 1] = offs[k] + *total;
}

// ================================================================ host

static inline unsigned blocks_for(int64_t items, int per_block) {
  int64_t b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (unsigned)b;
}

void configure_kernels() {
  cudaFuncSetAttribute(k_move_block<kBin3Threads, true>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kBin3Slots * (int)sizeof(unsigned long long));
}

void build_bins(const LevelGraph &g, Bins &b, int32_t *scan_tmp, cudaStream_t s) {
  cudaMemsetAsync(b.offs, 0, sizeof(int32_t), s);
  int64_t lo = -1;
  for (int k = 0; k < kBins; ++k) {
    const int64_t hi = k < kBins - 1 ? kBinMaxDeg[k] : INT64_MAX;
    scan_apply<int32_t>(g.n, BinFlag{g.rp, lo, hi}, BinEmit{b.lists, b.offs + k}, scan_tmp, s);
    k_bin_next_offset<<<1, 1, 0, s>>>(b.offs, k, scan_tmp + scan_tiles(g.n));
    lo = hi;
  }
}

void finish_bins(Bins &b, const int32_t *h_offs) {
  for (int k = 0; k < kBins; ++k) {
    b.list[k] = b.lists + h_offs[k];
    b.count[k] = h_offs[k + 1] - h_offs[k];
  }
}

template <int GS>
static void launch_vertex_kernel(void (*k)(PassArgs, const int32_t *, int64_t), const PassArgs &a,
                                 const int32_t *list, int64_t count, cudaStream_t s, size_t smem = 0) {
  if (count <= 0) return;
  const int threads = GS > 32 ? GS : 256;
  const int per_block = GS > 32 ? 1 : threads / GS;
  k<<<blocks_for(count, per_block), threads, smem, s>>>(a, list, count);
}

void launch_first_pass(const PassArgs &a, const Bins &b, cudaStream_t s) {
  launch_vertex_kernel<8>(k_first_pass<8>, a, b.list[0], b.count[0], s);
  launch_vertex_kernel<32>(k_first_pass<32>, a, b.list[1], b.count[1], s);
  launch_vertex_kernel<32>(k_first_pass<32>, a, b.list[2], b.count[2], s);
  launch_vertex_kernel<kBin3Threads>(k_first_pass<kBin3Threads>, a, b.list[3], b.count[3], s);
  launch_vertex_kernel<kBin4Threads>(k_first_pass<kBin4Threads>, a, b.list[4], b.count[4], s);
}

void launch_move(const PassArgs &a, const Bins &b, cudaStream_t s) {
  launch_vertex_kernel<8>(k_move_small<8>, a, b.list[0], b.count[0], s);
  launch_vertex_kernel<32>(k_move_small<32>, a, b.list[1], b.count[1], s);
  if (b.count[2] > 0)
    k_move_warp<<<blocks_for(b.count[2], kBin2Warps), kBin2Warps * 32, 0, s>>>(a, b.list[2],
                                                                              b.count[2]);
  launch_vertex_kernel<kBin3Threads>(k_move_block<kBin3Threads, true>, a, b.list[3], b.count[3], s,
                                     kBin3Slots * sizeof(unsigned long long));
  launch_vertex_kernel<kBin4Threads>(k_move_block<kBin4Threads, false>, a, b.list[4], b.count[4], s);
}

void launch_afterburner(const PassArgs &a, const Bins &b, cudaStream_t s) {
  launch_vertex_kernel<8>(k_afterburner<8>, a, b.list[0], b.count[0], s);
  launch_vertex_kernel<32>(k_afterburner<32>, a, b.list[1], b.count[1], s);
  launch_vertex_kernel<32>(k_afterburner<32>, a, b.list[2], b.count[2], s);
  launch_vertex_kernel<kBin3Threads>(k_afterburner<kBin3Threads>, a, b.list[3], b.count[3], s);
  launch_vertex_kernel<kBin4Threads>(k_afterburner<kBin4Threads>, a, b.list[4], b.count[4], s);
}

void launch_objective(const PassArgs &a, const Bins &b, cudaStream_t s) {
  launch_vertex_kernel<8>(k_objective<8>, a, b.list[0], b.count[0], s);
  launch_vertex_kernel<32>(k_objective<32>, a, b.list[1], b.count[1], s);
  launch_vertex_kernel<32>(k_objective<32>, a, b.list[2], b.count[2], s);
  launch_vertex_kernel<kBin3Threads>(k_objective<kBin3Threads>, a, b.list[3], b.count[3], s);
  launch_vertex_kernel<kBin4Threads>(k_objective<kBin4Threads>, a, b.list[4], b.count[4], s);
}

void launch_apply(const PassArgs &a, uint8_t *E, int32_t *used, int32_t *freelist,
                  int32_t *scan_tmp, cudaStream_t s) {
  k_apply<<<blocks_for(a.g.n, 256), 256, 0, s>>>(a, E);
  const int *k = &a.sc->empty_movers;
  k_zero_if<<<blocks_for(a.g.n, 256), 256, 0, s>>>(used, a.g.n, k);
  k_mark_occupied<<<blocks_for(a.g.n, 256), 256, 0, s>>>(a.C, E, used, a.g.n, k);
  scan_apply<int32_t>(a.g.n, FreeFlag{used}, FreeEmit{freelist, k}, scan_tmp, s, k);
  scan_apply<int32_t>(a.g.n, MoverFlag{E}, MoverEmit{freelist, a.C, a.W, a.g.vw, a.g.n, &a.sc->error}, scan_tmp, s, k);
}

void launch_pass_begin(Scalars *sc, cudaStream_t s) { k_pass_begin<<<1, 1, 0, s>>>(sc); }

void launch_bestof(Scalars *sc, const int32_t *C, int32_t *C_out, int64_t n, cudaStream_t s) {
  k_bestof_test<<<1, 1, 0, s>>>(sc);
  k_bestof_copy<<<blocks_for(n, 256), 256, 0, s>>>(sc, C, C_out, n);
}

void launch_iota(int32_t *C, int64_t n, cudaStream_t s) {
  k_iota<<<blocks_for(n, 256), 256, 0, s>>>(C, n);
}

void launch_cluster_weights(const int32_t *C, const int64_t *vw, int64_t *W, int64_t n,
                            cudaStream_t s) {
  cudaMemsetAsync(W, 0, sizeof(int64_t) * (size_t)(n > 0 ? n : 1), s);
  k_cluster_weights<<<blocks_for(n, 256), 256, 0, s>>>(C, vw, W, n);
}

}  // namespace lc
