// lc_pass.cu — kernels of one synchronous local-move pass (Algorithm 2 with
// the afterburner filter of Algorithm 3) and the per-level objective.
//
// Every vertex is handled by a thread group sized to its degree bin (see
// kBinMaxDeg in lc_internal.cuh).  The kernels are bound by the latency of
// dependent gathers (row offsets -> neighbours -> their clusters -> cluster
// weights), so each group issues its loads in batches before using them, and
// the bins keep many vertices in flight per SM.  Rows above 4096 entries
// ("hubs") are cut into chunks processed by independent blocks.
//
// All sums are integer (commutative atomics and shuffles), argmax ties go to
// the smallest cluster id and the afterburner order is a total order, so the
// results do not depend on scheduling.
#include <climits>

#include "lc_group.cuh"
#include "lc_internal.cuh"
#include "lc_pass.cuh"
#include "lc_scan.cuh"

namespace lc {

// ---------------------------------------------------- graphs of a batch

// Graph of vertex v in a packed batch (one graph: 0).
__device__ __forceinline__ int graph_of(const PassArgs &a, int32_t v) { return a.gid ? a.gid[v] : 0; }

// Records g(v, C[v]) for the objective: one graph accumulates in a register
// flushed once per block; a batch writes it per vertex and the per-graph
// sums are formed by k_graph_sums.
__device__ __forceinline__ void add_self(const PassArgs &a, int32_t v, long long gC, long long &phi) {
  if (a.gself)
    a.gself[v] = gC;
  else
    phi += gC;
}


// Kept tables: writes (X, S) into a table that only the calling thread
// touches (plain loads and stores; X is not in the table yet).  False if
// the table is full.
__device__ __forceinline__ bool tab_put(unsigned long long *t, uint32_t cap, int32_t X, long long S) {
  uint32_t s = slot_of(X, cap);
  for (uint32_t probe = 0; probe < cap; ++probe) {
    if (t[s] == kEmptySlot) {
      t[s] = ((unsigned long long)((uint32_t)X + 1u) << 32) | (uint32_t)S;
      return true;
    }
    s = (s + 1 == cap) ? 0 : s + 1;
  }
  return false;
}

// ---------------------------------------------------- vertex decision

// Algorithm 2 for one vertex once g(v, C[v]) and the best other cluster
// (gbest, best) are known: the empty-cluster rule, the candidate test with
// temperature phi = phi_n / phi_d, and delta_v (Algorithm 3's priority; its
// epsilon bucket is computed by k_ab_prep, off this latency-bound path).
__device__ __forceinline__ void decide(const PassArgs &a, const GraphParam &P, int32_t v, long long gC,
                                       int32_t best, long long gbest, long long &cntL) {
  if (!P.active) {  // graph not moving at this level (finished coarsening earlier)
    a.D[v] = kNone;
    return;
  }
  if (gC < 0 && (best == kNone || gbest < 0)) {
    best = kEmpty;
    gbest = 0;
  }
  const int32_t pn = a.phi_live ? a.phi_live[0] : a.phi_n;
  const int32_t pd = a.phi_live ? a.phi_live[1] : a.phi_d;
  const bool inL = best != kNone && (__int128)pd * gbest >= (__int128)(pd - pn) * (__int128)gC;
  if (inL) {
    a.D[v] = best;
    a.delta[v] = gbest - gC;
    cntL++;
  } else {
    a.D[v] = kNone;
  }
}

// ------------------------------------------- first pass (Section IV-A-3)

// Singleton start: the adjacent clusters of v are its neighbours, so the
// gains are read straight from the CSR: g(v,{u}) = Lam*w(u,v) - mu*w(v)*w(u),
// and g(v, C[v]) = 0.
__device__ __forceinline__ void first_edge(const PassArgs &a, const GraphParam &P, int64_t e,
                                           long long wv, long long &gb, int32_t &xb) {
  const int32_t u = __ldg(a.g.col + e);
  const long long g = P.Lam * (long long)__ldg(a.g.ew + e) - P.mu * wv * __ldg(a.g.vw + u);
  if (better(g, u, gb, xb)) {
    gb = g;
    xb = u;
  }
}

template <int GS>
__global__ void __launch_bounds__(GS > 32 ? GS : 256)
    k_first_pass(PassArgs a, const VRec *__restrict__ rec, int64_t count) {
  __shared__ long long rg[GS > 32 ? GS / 32 : 1];
  __shared__ int32_t rx[GS > 32 ? GS / 32 : 1];
  long long cntL = 0;
  const int r = Grp<GS>::rank();
  for_each_vertex<GS>(count, [&](int64_t i, bool active) {
    VRec vr{};
    if (active) vr = rec[i];
    const int32_t v = vr.v;
    const int64_t beg = vr.beg, end = vr.beg + vr.deg;
    const long long wv = vr.w;
    const GraphParam P = a.gp[vr.g];
    long long gb = LLONG_MIN;
    int32_t xb = kNone;
#pragma unroll 4
    for (int64_t e = beg + r; e < end; e += GS) first_edge(a, P, e, wv, gb, xb);
    Grp<GS>::argmax(gb, xb, rg, rx);
    if (active && r == 0) decide(a, P, v, 0, xb, gb, cntL);
  });
  flush_block_sum(cntL, &a.sc->count_L);
}

// ----------------------------------- aggregation + argmax, bin 0 (thread)

// One thread per vertex of degree <= 8: neighbour clusters and weights are
// held in registers; S(v, X) for each distinct X is an unrolled compare-sum.
__global__ void __launch_bounds__(256, 4) k_move_thread(PassArgs a, const VRec *__restrict__ rec,
                                                        int64_t count) {
  constexpr int K = 8;
  long long cntL = 0, phi = 0, nX = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const VRec vr = rec[i];
    const int32_t v = vr.v;
    const int64_t beg = vr.beg;
    const int deg = vr.deg;
    const int32_t Cv = LC_IDX(a.C[v], a.g.n, kDbgLabel);
    const long long wv = vr.w;
    const GraphParam P = a.gp[vr.g];
    int32_t u[K], w[K], X[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      u[j] = 0;
      w[j] = 0;
      if (j < deg) {
        u[j] = LC_IDX(__ldg(a.g.col + beg + j), a.g.n, kDbgColumn);
        w[j] = __ldg(a.g.ew + beg + j);
      }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) X[j] = j < deg ? LC_IDX(a.C[u[j]], a.g.n, kDbgLabel) : -1;
    const long long WC = a.W[Cv];
    long long WX[K];
#pragma unroll
    for (int j = 0; j < K; ++j) WX[j] = (j < deg && X[j] != Cv) ? a.W[X[j]] : 0;
    long long self = 0, gb = LLONG_MIN;
    int32_t xb = kNone;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (j >= deg) continue;
      if (X[j] == Cv) {
        self += w[j];
        continue;
      }
      bool first = true;
      long long S = 0;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (k < deg && X[k] == X[j]) {
          S += w[k];
          if (k < j) first = false;
        }
      }
      if (first) {
        nX++;
        const long long g = gain_other(P, S, wv, WX[j]);
        if (better(g, X[j], gb, xb)) {
          gb = g;
          xb = X[j];
        }
      }
    }
    const long long gC = gain_self(P, self, wv, WC);
    add_self(a, v, gC, phi);
    decide(a, P, v, gC, xb, gb, cntL);
  }
  flush_block_sum(nX, &a.sc->distinct_x);
  flush_block_sum(cntL, &a.sc->count_L);
  flush_block_sum(phi, &a.phi_acc[0]);
}

// ------------------------------------ aggregation + argmax, bins 1-2 (lanes)

// Each lane holds one neighbour; lanes of a group with the same neighbour
// cluster are matched with __match_any_sync and their weights summed in a
// per-lane shared slot of the lowest matching lane.  S(v, C[v]) is a group
// reduction (the dedicated current-cluster slot of Section IV-A-3).
template <int G>
__global__ void __launch_bounds__(256) k_move_small(PassArgs a, const VRec *__restrict__ rec,
                                                    int64_t count) {
  static_assert(G == 16 || G == 32, "the match key holds one group bit");
  __shared__ int32_t acc[256];
  long long cntL = 0, phi = 0, nX = 0;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (G - 1);
  const int wbase = threadIdx.x & ~31;
  for_each_vertex<G>(count, [&](int64_t i, bool active) {
    VRec vr{};
    if (active) vr = rec[i];
    const int32_t v = vr.v;
    const int64_t beg = vr.beg, deg = vr.deg;
    const int32_t Cv = active ? LC_IDX(a.C[v], a.g.n, kDbgLabel) : 0;
    const long long wv = vr.w;
    const GraphParam P = a.gp[vr.g];
    const bool has = sub < deg;
    int32_t X = -1, w = 0;
    if (has) {
      const int32_t u = LC_IDX(__ldg(a.g.col + beg + sub), a.g.n, kDbgColumn);
      w = __ldg(a.g.ew + beg + sub);
      X = LC_IDX(a.C[u], a.g.n, kDbgLabel);
    }
    const long long WC = (active && sub == 0) ? a.W[Cv] : 0;
    const bool self = has && X == Cv;
    const bool other = has && !self;
    const long long WX = other ? a.W[X] : 0;
    const long long S_self = group_sum<G>((long long)(self ? w : 0));
    // 32-bit match key: the lane's group in bit 31 (G = 16) above the
    // cluster id (< 2^31 - 1); lanes with nothing to add share the key
    // 0xFFFFFFFF, which no (group, cluster) pair takes, and never add
    const uint32_t key = other ? ((G < 32 ? (uint32_t)(lane / G) << 31 : 0u) | (uint32_t)X) : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
    const int leader = __ffs(peers) - 1;
    acc[threadIdx.x] = 0;
    __syncwarp();
    if (other) atomicAdd(&acc[wbase + leader], w);
    __syncwarp();
    long long g = LLONG_MIN;
    int32_t x = kNone;
    if (other && lane == leader) {
      g = gain_other(P, acc[threadIdx.x], wv, WX);
      x = X;
      nX++;
    }
    group_argmax<G>(g, x);
    if (active && sub == 0) {
      const long long gC = gain_self(P, S_self, wv, WC);
      add_self(a, v, gC, phi);
      decide(a, P, v, gC, x, g, cntL);
    }
    __syncwarp();
  });
  flush_block_sum(nX, &a.sc->distinct_x);
  flush_block_sum(cntL, &a.sc->count_L);
  flush_block_sum(phi, &a.phi_acc[0]);
}

// ------------------------------------ shared-table aggregation, bins 3-5

// Shared tables stay clean between vertices: a vertex's argmax scans the
// slots [0, cap) it may have used and resets the occupied ones.  The warp
// bins use 2 deg rounded up to 32 slots (load <= 1/2, whole warps of slots);
// the block bins use tab_cap(deg), the layout of the kept tables.
__device__ __forceinline__ uint32_t warp_table_cap(int64_t deg) {
  return (uint32_t)((2 * deg + 31) & ~31ll);
}

// Best (gain, cluster) over slots [s0, s1) of a table (strided by GS),
// resetting the slots it reads unless `keep` (a kept table being built).
// g(v, X) = Lam S(v, X) - (mu w(v)) W(X), with mu w(v) formed once.
template <int GS>
__device__ __forceinline__ void range_argmax(const PassArgs &a, const GraphParam &P,
                                             unsigned long long *tab, uint32_t s0, uint32_t s1,
                                             long long wv, int r, long long &gb, int32_t &xb,
                                             long long &nX, bool keep = false) {
  constexpr int U = 4;
  const long long Lam = P.Lam, muw = P.mu * wv;
  for (uint32_t base = s0 + r; base < s1; base += GS * U) {
    unsigned long long t[U];
    long long WX[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const uint32_t s = base + k * GS;
      t[k] = s < s1 ? tab[s] : kEmptySlot;
      if (t[k] != kEmptySlot && !keep) tab[s] = kEmptySlot;
    }
#pragma unroll
    for (int k = 0; k < U; ++k) WX[k] = t[k] != kEmptySlot ? a.W[LC_IDX(slot_key(t[k]), a.g.n, kDbgLabel)] : 0;
#pragma unroll
    for (int k = 0; k < U; ++k) {
      if (t[k] == kEmptySlot) continue;
      nX++;
      const int32_t X = slot_key(t[k]);
      const long long g = Lam * (long long)slot_val(t[k]) - muw * WX[k];
      if (better(g, X, gb, xb)) {
        gb = g;
        xb = X;
      }
    }
  }
}

// ------------------------------ split shared tables (warp and block bins)

// A shared table kept as two 32-bit arrays: key[s] (0 = empty, else the
// cluster id + 1) and val[s] (the weight sum S(v, X)).  Claiming a slot is
// a 32-bit CAS on the key and every edge then adds its weight with a 32-bit
// atomic add, which shared memory executes far faster than 64-bit CAS.
struct SplitTab {
  uint32_t *key;
  int32_t *val;
};

// Sequential probing from slot s for cluster X (tag = X + 1).
__device__ __forceinline__ bool split_probe(SplitTab t, uint32_t cap, uint32_t tag, int32_t w,
                                            uint32_t s) {
  for (uint32_t probe = 0; probe < cap; ++probe) {
    uint32_t k = t.key[s];
    if (k == 0u) k = atomicCAS(&t.key[s], 0u, tag);
    if (k == 0u || k == tag) {
      atomicAdd(&t.val[s], w);
      return true;
    }
    s = (s + 1 == cap) ? 0 : s + 1;
  }
  return false;
}

// Adds (X[k], w[k]) for every k with todo[k]: the first probe of all U
// entries is read at once; a slot holding the key takes the weight, an
// empty one is claimed by CAS (a CAS that finds the key takes it too), and
// only a slot holding another key falls back to sequential probing.
template <int U>
__device__ __forceinline__ void split_add_batch(SplitTab t, uint32_t cap, const int32_t (&X)[U],
                                                const int32_t (&w)[U], const bool (&todo)[U],
                                                bool &ok) {
  uint32_t sl[U], cur[U];
#pragma unroll
  for (int k = 0; k < U; ++k) {
    sl[k] = todo[k] ? slot_of(X[k], cap) : 0;
    cur[k] = todo[k] ? t.key[sl[k]] : 0;
  }
#pragma unroll
  for (int k = 0; k < U; ++k)
    if (todo[k] && cur[k] == 0u) cur[k] = atomicCAS(&t.key[sl[k]], 0u, (uint32_t)X[k] + 1u);
#pragma unroll
  for (int k = 0; k < U; ++k) {
    if (!todo[k]) continue;
    const uint32_t tag = (uint32_t)X[k] + 1u;
    if (cur[k] == 0u || cur[k] == tag)
      atomicAdd(&t.val[sl[k]], w[k]);
    else
      ok &= split_probe(t, cap, tag, w[k], sl[k] + 1 == cap ? 0 : sl[k] + 1);
  }
}

// Inserts edges [beg, end) of v (strided by GS, U edges per thread at a
// time).  Returns this thread's part of S(v, C[v]).  Indices are
// row-relative 32-bit (a row has fewer than 2^31 entries).
template <int GS, int U>
__device__ __forceinline__ long long split_insert_row(const PassArgs &a, int64_t beg, int64_t end,
                                                      int32_t Cv, SplitTab t, uint32_t cap, int r,
                                                      bool &ok) {
  const int32_t *__restrict__ col = a.g.col + beg;
  const int32_t *__restrict__ ew = a.g.ew + beg;
  const int deg = (int)(end - beg);
  long long self = 0;
  for (int base = r; base < deg; base += GS * U) {
    int32_t u[U], w[U], X[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int e = base + k * GS;
      u[k] = -1;
      w[k] = 0;
      if (e < deg) {
        u[k] = LC_IDX(__ldg(col + e), a.g.n, kDbgColumn);
        w[k] = __ldg(ew + e);
      }
    }
#pragma unroll
    for (int k = 0; k < U; ++k) X[k] = u[k] >= 0 ? LC_IDX(a.C[u[k]], a.g.n, kDbgLabel) : -1;
    bool todo[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      todo[k] = u[k] >= 0 && X[k] != Cv;
      if (u[k] >= 0 && X[k] == Cv) self += w[k];
    }
    split_add_batch<U>(t, cap, X, w, todo, ok);
  }
  return self;
}

// Best (gain, cluster) over slots [0, cap) (strided by GS), resetting the
// occupied ones.  g(v, X) = Lam S(v, X) - (mu w(v)) W(X).  BUILD: every
// slot is also copied to the kept table gt (same layout, empties included).
template <int GS, bool BUILD>
__device__ __forceinline__ void split_argmax(const PassArgs &a, const GraphParam &P, SplitTab t,
                                             uint32_t cap, long long wv, int r, long long &gb,
                                             int32_t &xb, unsigned long long *gt, long long &nX) {
  constexpr int U = 4;
  const long long Lam = P.Lam, muw = P.mu * wv;
  for (uint32_t base = r; base < cap; base += GS * U) {
    uint32_t key[U];
    int32_t S[U];
    long long WX[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const uint32_t s = base + k * GS;
      key[k] = s < cap ? t.key[s] : 0u;
      S[k] = 0;
      if (key[k] != 0u) {
        S[k] = t.val[s];
        t.key[s] = 0u;
        t.val[s] = 0;
      }
    }
    if constexpr (BUILD) {
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const uint32_t s = base + k * GS;
        if (s < cap) gt[s] = key[k] != 0u ? ((unsigned long long)key[k] << 32) | (uint32_t)S[k] : kEmptySlot;
      }
    }
#pragma unroll
    for (int k = 0; k < U; ++k) WX[k] = key[k] != 0u ? a.W[LC_IDX(key[k] - 1u, a.g.n, kDbgLabel)] : 0;
#pragma unroll
    for (int k = 0; k < U; ++k) {
      if (key[k] == 0u) continue;
      nX++;
      const int32_t X = (int32_t)(key[k] - 1u);
      const long long g = Lam * (long long)S[k] - muw * WX[k];
      if (better(g, X, gb, xb)) {
        gb = g;
        xb = X;
      }
    }
  }
}

// Bins 3-4: one warp per vertex, a per-warp split shared table of SLOTS
// slots.
template <int SLOTS>
__global__ void __launch_bounds__(kWarpBinWarps * 32, 4)
    k_move_warp(PassArgs a, const VRec *__restrict__ rec, int64_t count) {
  constexpr int U = SLOTS / 128;  // edges per lane per batch: 64 (bin 3) or 128 (bin 4)
  __shared__ uint32_t keys[kWarpBinWarps][SLOTS];
  __shared__ int32_t vals[kWarpBinWarps][SLOTS];
  long long cntL = 0, phi = 0, nX = 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const SplitTab tab{keys[wid], vals[wid]};
  for (int s = lane; s < SLOTS; s += 32) {
    tab.key[s] = 0u;
    tab.val[s] = 0;
  }
  __syncwarp();
  for_each_vertex<32>(count, [&](int64_t i, bool active) {
    if (!active) return;  // warp-uniform: the whole warp shares i
    const VRec vr = rec[i];
    const int32_t v = vr.v;
    const int64_t beg = vr.beg, end = vr.beg + vr.deg;
    const int32_t Cv = LC_IDX(a.C[v], a.g.n, kDbgLabel);
    const long long wv = vr.w;
    const GraphParam P = a.gp[vr.g];
    const uint32_t cap = warp_table_cap(end - beg);
    bool ok = true;
    long long self = split_insert_row<32, U>(a, beg, end, Cv, tab, cap, lane, ok);
    if (!ok) {
      a.sc->error = 1;
      LC_DBG_FAIL(kDbgProbe, v, a.g.n);
    }
    const long long WC = lane == 0 ? a.W[Cv] : 0;
    __syncwarp();
    long long gb = LLONG_MIN;
    int32_t xb = kNone;
    split_argmax<32, false>(a, P, tab, cap, wv, lane, gb, xb, nullptr, nX);
    group_argmax<32>(gb, xb);
    self = warp_sum(self);
    if (lane == 0) {
      const long long gC = gain_self(P, self, wv, WC);
      add_self(a, v, gC, phi);
      decide(a, P, v, gC, xb, gb, cntL);
    }
    __syncwarp();
  });
  flush_block_sum(nX, &a.sc->distinct_x);
  flush_block_sum(cntL, &a.sc->count_L);
  flush_block_sum(phi, &a.phi_acc[0]);
}

// Bins 5-8: one block per vertex; dynamic shared memory holds the split
// table (SLOTS keys, then SLOTS values).  A row uses min(2 deg rounded up
// to 32, SLOTS) slots: bin 8 (deg <= 4096) has 6144 slots, a load factor of
// at most 2/3, so that four blocks fit in an SM's shared memory.
// BUILD: the tables use the kept-table layout (tab_cap slots) and are
// copied out to each vertex's gtab region with S(v, C[v]) added.
template <int GS, int SLOTS, bool BUILD>
__global__ void __launch_bounds__(GS) k_move_block(PassArgs a, const VRec *__restrict__ rec,
                                                   int64_t count) {
  extern __shared__ uint32_t smem_tab[];
  const SplitTab tab{smem_tab, reinterpret_cast<int32_t *>(smem_tab + SLOTS)};
  // per-warp partials, double-buffered by vertex parity: thread 0 combines
  // vertex i's while the other threads already insert vertex i + 1, and the
  // buffer is written again only after two more barriers (vertex i + 2)
  __shared__ long long rs[2][GS / 32];
  __shared__ long long rg[2][GS / 32];
  __shared__ int32_t rx[2][GS / 32];
  int par = 0;
  long long cntL = 0, phi = 0, nX = 0;
  for (int s = threadIdx.x; s < SLOTS; s += GS) {
    tab.key[s] = 0u;
    tab.val[s] = 0;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
    const VRec vr = rec[i];
    const int32_t v = vr.v;
    const int64_t beg = vr.beg, end = vr.beg + vr.deg;
    const int32_t Cv = LC_IDX(a.C[v], a.g.n, kDbgLabel);
    const long long wv = vr.w;
    const GraphParam P = a.gp[vr.g];
    const uint32_t cap = BUILD ? tab_cap(end - beg) : min(warp_table_cap(end - beg), (uint32_t)SLOTS);
    bool ok = true;
    long long self = split_insert_row<GS, 4>(a, beg, end, Cv, tab, cap, threadIdx.x, ok);
    if (!ok) {
      a.sc->error = 1;
      LC_DBG_FAIL(kDbgProbe, v, a.g.n);
    }
    const long long WC = threadIdx.x == 0 ? a.W[Cv] : 0;
    __syncthreads();
    long long gb = LLONG_MIN;
    int32_t xb = kNone;
    unsigned long long *gt = a.gtab + 2 * beg;
    split_argmax<GS, BUILD>(a, P, tab, cap, wv, threadIdx.x, gb, xb, gt, nX);
    // one reduction of (best gain, cluster, S_self) for thread 0 only: warp
    // level, one barrier, thread 0 combines the warps
    group_argmax<32>(gb, xb);
    self = warp_sum(self);
    if ((threadIdx.x & 31) == 0) {
      rg[par][threadIdx.x >> 5] = gb;
      rx[par][threadIdx.x >> 5] = xb;
      rs[par][threadIdx.x >> 5] = self;
    }
    // the table is read and reset by every thread past this barrier, so the
    // next vertex may start inserting at once
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < GS / 32; ++w) {
        self += rs[par][w];
        if (better(rg[par][w], rx[par][w], gb, xb)) {
          gb = rg[par][w];
          xb = rx[par][w];
        }
      }
      // the barrier above made every thread's copied slots visible
      if (BUILD && self > 0 && !tab_put(gt, cap, Cv, self)) a.sc->error = 1;
      const long long gC = gain_self(P, self, wv, WC);
      add_self(a, v, gC, phi);
      decide(a, P, v, gC, xb, gb, cntL);
    }
    par ^= 1;
  }
  flush_block_sum(nX, &a.sc->distinct_x);
  flush_block_sum(cntL, &a.sc->count_L);
  flush_block_sum(phi, &a.phi_acc[0]);
}

// --------------------------------------------------------- hubs (bin 9)

// Block-wide argmax of (g, x) into the chunk partials.
__device__ __forceinline__ void hub_part_store(const PassArgs &a, int c, long long gb, int32_t xb) {
  __shared__ long long rg[kHubThreads / 32];
  __shared__ int32_t rx[kHubThreads / 32];
  Grp<kHubThreads>::argmax(gb, xb, rg, rx);
  if (threadIdx.x == 0) {
    a.hub.part_g[c] = gb;
    a.hub.part_x[c] = xb;
  }
}

__device__ __forceinline__ void hub_acc_add(const PassArgs &a, int h, long long x) {
  __shared__ long long rs[kHubThreads / 32];
  x = Grp<kHubThreads>::sum(x, rs);
  if (threadIdx.x == 0 && x != 0) atomicAdd((unsigned long long *)&a.hub.acc[h], (unsigned long long)x);
}

// Move, step 1: insert a chunk of a hub row into the hub's global table.
// Lanes of a warp holding the same cluster are combined first
// (__match_any_sync), so a popular cluster costs one global atomic per warp.
__global__ void __launch_bounds__(kHubThreads) k_hub_move_insert(PassArgs a) {
  constexpr int U = 4;
  __shared__ int32_t acc[kHubThreads];
  const int c = blockIdx.x;
  const int h = a.hub.hub_of[c];
  const int32_t v = a.hub.vtx[h];
  const int64_t beg = a.g.rp[v], end = a.g.rp[v + 1];
  const int32_t Cv = LC_IDX(a.C[v], a.g.n, kDbgLabel);
  unsigned long long *tab = a.gtab + 2 * beg;
  const uint32_t cap = (uint32_t)(2 * (end - beg));
  const int lane = threadIdx.x & 31, wbase = threadIdx.x & ~31;
  const int64_t e0 = a.hub.e0[c], e1 = a.hub.e1[c];
  long long self = 0;
  bool ok = true;
  for (int64_t base = e0; base < e1; base += kHubThreads * U) {
    int32_t u[U], w[U], X[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int64_t e = base + k * kHubThreads + threadIdx.x;
      u[k] = -1;
      w[k] = 0;
      if (e < e1) {
        u[k] = LC_IDX(__ldg(a.g.col + e), a.g.n, kDbgColumn);
        w[k] = __ldg(a.g.ew + e);
      }
    }
#pragma unroll
    for (int k = 0; k < U; ++k) X[k] = u[k] >= 0 ? LC_IDX(a.C[u[k]], a.g.n, kDbgLabel) : -1;
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const bool other = u[k] >= 0 && X[k] != Cv;
      if (u[k] >= 0 && X[k] == Cv) self += w[k];
      // lanes with nothing to add share the key 0xFFFFFFFF (no cluster id)
      const uint32_t key = other ? (uint32_t)X[k] : 0xFFFFFFFFu;
      const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
      const int leader = __ffs(peers) - 1;
      acc[threadIdx.x] = 0;
      __syncwarp();
      if (other) atomicAdd(&acc[wbase + leader], w[k]);
      __syncwarp();
      if (other && lane == leader) {
        bool fresh = false;
        ok &= table_add(tab, cap, X[k], acc[threadIdx.x], fresh);
      }
      __syncwarp();
    }
  }
  if (!ok) {
    a.sc->error = 1;
    LC_DBG_FAIL(kDbgProbe, v, a.g.n);
  }
  hub_acc_add(a, h, self);
}

// Move, step 2: argmax over the chunk's share of the hub table (reset as
// read, or kept as the hub's kept table with a.tab_build).
__global__ void __launch_bounds__(kHubThreads) k_hub_move_scan(PassArgs a) {
  const int c = blockIdx.x;
  const int h = a.hub.hub_of[c];
  const int32_t v = a.hub.vtx[h];
  const int64_t beg = a.g.rp[v];
  const long long wv = a.g.vw[v];
  const GraphParam P = a.gp[graph_of(a, v)];
  long long gb = LLONG_MIN, nX = 0;
  int32_t xb = kNone;
  range_argmax<kHubThreads>(a, P, a.gtab + 2 * beg, (uint32_t)(2 * (a.hub.e0[c] - beg)),
                            (uint32_t)(2 * (a.hub.e1[c] - beg)), wv, threadIdx.x, gb, xb, nX,
                            a.tab_build != 0);
  hub_part_store(a, c, gb, xb);
  flush_block_sum(nX, &a.sc->distinct_x);
}

// First pass: argmax over a chunk of a hub row.
__global__ void __launch_bounds__(kHubThreads) k_hub_first(PassArgs a) {
  const int c = blockIdx.x;
  const int32_t v = a.hub.vtx[a.hub.hub_of[c]];
  const long long wv = a.g.vw[v];
  const GraphParam P = a.gp[graph_of(a, v)];
  long long gb = LLONG_MIN;
  int32_t xb = kNone;
#pragma unroll 4
  for (int64_t e = a.hub.e0[c] + threadIdx.x; e < a.hub.e1[c]; e += kHubThreads)
    first_edge(a, P, e, wv, gb, xb);
  hub_part_store(a, c, gb, xb);
}

// Final step per hub: combine chunk partials, then decide (Algorithm 2).
// first = 1: singleton start, g(v, C[v]) = 0 and no objective term.
__global__ void k_hub_decide(PassArgs a, int first) {
  long long cntL = 0, phi = 0;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < a.hub.H; h += gridDim.x * blockDim.x) {
    const int32_t v = a.hub.vtx[h];
    const GraphParam P = a.gp[graph_of(a, v)];
    long long gb = LLONG_MIN;
    int32_t xb = kNone;
    for (int c = a.hub.c0[h]; c < a.hub.c0[h + 1]; ++c)
      if (better(a.hub.part_g[c], a.hub.part_x[c], gb, xb)) {
        gb = a.hub.part_g[c];
        xb = a.hub.part_x[c];
      }
    long long gC = 0;
    if (!first) {
      const long long self = a.hub.acc[h];
      a.hub.acc[h] = 0;
      const int32_t Cv = a.C[v];
      gC = gain_self(P, self, a.g.vw[v], a.W[Cv]);
      add_self(a, v, gC, phi);
      if (a.tab_build && self > 0) {  // the hub's kept table gets its own cluster
        const int64_t beg = a.g.rp[v];
        if (!tab_put(a.gtab + 2 * beg, tab_cap(a.g.rp[v + 1] - beg), Cv, self)) a.sc->error = 1;
      }
    }
    decide(a, P, v, gC, xb, gb, cntL);
  }
  flush_block_sum(cntL, &a.sc->count_L);
  flush_block_sum(phi, &a.phi_acc[0]);
}

// ------------------------------------------------ afterburner (Algorithm 3)

// Packs {C, D, epsilon bucket of delta} per candidate for the afterburner's
// neighbour gathers (one 16-byte load each).  The bucket of Section IV-A-1,
// floor(eps_den * delta / (eps_num * Lambda)), needs a 128-bit division; it
// is done here, one thread per vertex, off the aggregation kernels.
// It also writes the candidate bitmap (one ballot per warp: a warp covers 32
// consecutive, aligned ids), lists the candidates below the hub degree by
// afterburner group (warp-aggregated appends; the order inside a list does
// not matter, each candidate's sum is independent of the others), clears
// M, and sums the candidates' degrees (the afterburner's edge work) into
// sc->cand_edges for the algorithmic-byte count of the profile.
__global__ void __launch_bounds__(256) k_ab_prep(PassArgs a) {
  long long cand = 0;
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.g.n;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = base + threadIdx.x;
    const int64_t w0 = base + (threadIdx.x & ~31);  // first id of this warp
    bool isc = false;
    int grp = -1;
    AbWork wk;
    if (v < a.g.n) {
      AbRec r;
      r.D = a.D[v];
      isc = r.D != kNone;
      a.M[v] = 0;  // survivors are set by the afterburner kernels
      if (isc) {
        // only candidates' records are ever read (the bitmap filters the
        // neighbour gathers, hubs read their own only as candidates)
        r.C = a.C[v];
        const GraphParam P = a.gp[graph_of(a, (int32_t)v)];
        const long long dv = a.delta[v];
        r.q = eps_bucket(a.m, P.Lam, dv);
        a.ab[v] = r;
        const int64_t beg = a.g.rp[v];
        const int64_t deg = a.g.rp[v + 1] - beg;
        cand += deg;
        for (int k = 0; k < kAbGroups && grp < 0; ++k)
          if (deg <= a.ab_max[k]) grp = k;  // hubs stay unlisted (grp -1)
        wk.v = (int32_t)v;
        wk.C = r.C;
        wk.D = r.D;
        wk.deg = (int32_t)deg;
        wk.vbase = P.vbase;
        wk.hv = fmix32((uint32_t)((int32_t)v - P.vbase) ^ a.m.seed);  // the id within its graph
        wk.q = r.q;
        wk.muw = P.mu * a.g.vw[v];
        wk.Lam = P.Lam;
        wk.beg = beg;
        wk.delta = dv;
      }
    }
    const unsigned bits = __ballot_sync(0xFFFFFFFFu, isc);
    if (lane == 0 && w0 < a.g.n) a.inL[w0 >> 5] = bits;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, grp);
    if (grp >= 0) {
      const int leader = __ffs(peers) - 1;
      int pos = 0;
      if (lane == leader) pos = atomicAdd(&a.sc->ab_count[grp], __popc(peers));
      pos = __shfl_sync(peers, pos, leader) + __popc(peers & ((1u << lane) - 1u));
      a.ab_list[a.ab_off[grp] + pos] = wk;
    }
  }
  flush_block_sum(cand, &a.sc->cand_edges);
}

struct AbCtx {
  int32_t v, Cv, Dv, vbase;
  long long qv, muw, Lam;
  uint32_t hv;
};

// A hub's context, gathered (hubs are not listed with work records).
__device__ __forceinline__ AbCtx ab_ctx(const PassArgs &a, int32_t v) {
  const AbRec r = a.ab[v];
  AbCtx c;
  c.v = v;
  c.Cv = r.C;
  c.Dv = r.D;
  c.qv = r.q;
  const GraphParam P = a.gp[graph_of(a, v)];
  c.vbase = P.vbase;
  c.muw = P.mu * a.g.vw[v];
  c.Lam = P.Lam;
  // the hash takes the id within the vertex's own graph
  c.hv = fmix32((uint32_t)(v - c.vbase) ^ a.m.seed);
  return c;
}

__device__ __forceinline__ AbCtx ab_ctx(const AbWork &w) {
  AbCtx c;
  c.v = w.v;
  c.Cv = w.C;
  c.Dv = w.D;
  c.qv = w.q;
  c.vbase = w.vbase;
  c.muw = w.muw;
  c.Lam = w.Lam;
  c.hv = w.hv;
  return c;
}

// Sum over edges [e0, e1) (strided by GS, loads batched U at a time) of the
// change of v's two gains when an adjacent candidate u that precedes v moves
// from C[u] to D[u] (Algorithm 3's four rules).
template <int GS, int U>
__device__ __forceinline__ long long ab_edges(const PassArgs &a, const AbCtx &c, int64_t e0,
                                              int64_t e1, int r) {
  long long d = 0;
  const int32_t *__restrict__ col = a.g.col + e0;
  const int32_t *__restrict__ ew = a.g.ew + e0;
  const int len = (int)(e1 - e0);
  const long long muw = c.muw;
  for (int base = r; base < len; base += GS * U) {
    int32_t u[U], w[U];
    AbRec rec[U];
    long long wu[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int e = base + k * GS;
      u[k] = -1;
      w[k] = 0;
      if (e < len) {
        u[k] = LC_IDX(__ldg(col + e), a.g.n, kDbgColumn);
        w[k] = __ldg(ew + e);
      }
    }
    // only candidates matter (Algorithm 3): test the bitmap first, gather
    // the 16-byte record of candidate neighbours only
    uint32_t word[U];
#pragma unroll
    for (int k = 0; k < U; ++k) word[k] = u[k] >= 0 ? __ldg(a.inL + (u[k] >> 5)) : 0u;
#pragma unroll
    for (int k = 0; k < U; ++k) {
      rec[k].D = kNone;
      if ((word[k] >> (u[k] & 31)) & 1u) rec[k] = a.ab[u[k]];
    }
    bool need[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      need[k] = rec[k].D != kNone &&
                (rec[k].q != c.qv ? rec[k].q > c.qv
                                  : earlier(rec[k].q, fmix32((uint32_t)(u[k] - c.vbase) ^ a.m.seed),
                                            u[k], c.qv, c.hv, c.v));
      wu[k] = need[k] ? a.g.vw[u[k]] : 0;
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      if (!need[k]) continue;
      const long long aw = c.Lam * (long long)w[k] - muw * wu[k];
      const int32_t Cu = rec[k].C, Du = rec[k].D;
      if (c.Cv == Cu)
        d += aw;
      else if (c.Dv == Cu)
        d -= aw;
      if (c.Cv == Du)
        d -= aw;
      else if (c.Dv >= 0 && c.Dv == Du)
        d += aw;
    }
  }
  return d;
}

// For each candidate v: delta_v adjusted by every adjacent candidate u that
// precedes v in the order; v survives iff the adjusted delta is >= 0.
// list / *count: the candidates of one group, listed by k_ab_prep.
template <int GS>
__global__ void __launch_bounds__(GS > 32 ? GS : 256, GS > 32 ? 2048 / GS / 2 : 4)
    k_afterburner(PassArgs a, const AbWork *__restrict__ list, const int *__restrict__ count_ptr) {
  constexpr int U = 4;
  long long cntM = 0;
  const int r = Grp<GS>::rank();
  const int64_t count = *count_ptr;
  if constexpr (GS > 32) {
    // block per candidate: the per-warp sums alternate between two buffers,
    // so one barrier per candidate suffices (the next candidate's barrier
    // orders thread 0's reads before the buffer is written again)
    __shared__ long long rs[2][GS / 32];
    int par = 0;
    for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
      const AbWork wk = list[i];
      const AbCtx c = ab_ctx(wk);
      long long acc = warp_sum(ab_edges<GS, U>(a, c, wk.beg, wk.beg + wk.deg, r));
      if ((threadIdx.x & 31) == 0) rs[par][threadIdx.x >> 5] = acc;
      __syncthreads();
      if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < GS / 32; ++w) t += rs[par][w];
        const bool keep = wk.delta + t >= 0;
        a.M[wk.v] = keep;
        cntM += keep;
      }
      par ^= 1;
    }
  } else {
    __shared__ long long rs[1];
    for_each_vertex<GS>(count, [&](int64_t i, bool active) {
      AbWork wk;
      long long acc = 0;
      if (active) {
        wk = list[i];
        const AbCtx c = ab_ctx(wk);
        acc = ab_edges<GS, U>(a, c, wk.beg, wk.beg + wk.deg, r);
      }
      acc = Grp<GS>::sum(acc, rs);
      if (active && r == 0) {
        const bool keep = wk.delta + acc >= 0;
        a.M[wk.v] = keep;
        cntM += keep;
      }
    });
  }
  flush_block_sum(cntM, &a.sc->count_M);
}

__global__ void __launch_bounds__(kHubThreads) k_hub_afterburner(PassArgs a) {
  const int c = blockIdx.x;
  const int h = a.hub.hub_of[c];
  const int32_t v = a.hub.vtx[h];
  if (a.D[v] == kNone) return;  // block-uniform
  const AbCtx ctx = ab_ctx(a, v);
  const long long acc = ab_edges<kHubThreads, 4>(a, ctx, a.hub.e0[c], a.hub.e1[c], threadIdx.x);
  hub_acc_add(a, h, acc);
}

__global__ void k_hub_ab_final(PassArgs a) {
  long long cntM = 0;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < a.hub.H; h += gridDim.x * blockDim.x) {
    const int32_t v = a.hub.vtx[h];
    const long long acc = a.hub.acc[h];
    a.hub.acc[h] = 0;
    const bool keep = a.D[v] != kNone && a.delta[v] + acc >= 0;
    a.M[v] = keep;
    cntM += keep;
  }
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
#pragma unroll 4
      for (int64_t e = beg + r; e < end; e += GS)
        if (a.C[LC_IDX(__ldg(a.g.col + e), a.g.n, kDbgColumn)] == Cv) self += __ldg(a.g.ew + e);
    }
    self = Grp<GS>::sum(self, rs);
    if (active && r == 0)
      add_self(a, v, gain_self(a.gp[graph_of(a, v)], self, a.g.vw[v], a.W[Cv]), phi);
  });
  flush_block_sum(phi, &a.phi_acc[0]);
}

__global__ void __launch_bounds__(kHubThreads) k_hub_objective(PassArgs a) {
  const int c = blockIdx.x;
  const int h = a.hub.hub_of[c];
  const int32_t Cv = a.C[a.hub.vtx[h]];
  long long self = 0;
#pragma unroll 4
  for (int64_t e = a.hub.e0[c] + threadIdx.x; e < a.hub.e1[c]; e += kHubThreads)
    if (a.C[LC_IDX(__ldg(a.g.col + e), a.g.n, kDbgColumn)] == Cv) self += __ldg(a.g.ew + e);
  hub_acc_add(a, h, self);
}

__global__ void k_hub_obj_final(PassArgs a) {
  long long phi = 0;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < a.hub.H; h += gridDim.x * blockDim.x) {
    const int32_t v = a.hub.vtx[h];
    const long long self = a.hub.acc[h];
    a.hub.acc[h] = 0;
    add_self(a, v, gain_self(a.gp[graph_of(a, v)], self, a.g.vw[v], a.W[a.C[v]]), phi);
  }
  flush_block_sum(phi, &a.phi_acc[0]);
}

// ------------------------------------------ kept tables (Section IV-A-3)
//
// Vertices of degree above kTabMinDeg (bins 5-9) may keep their S(v, .)
// across the passes of one LocalMovePasses call.  An aggregation pass with
// a.tab_build copies each block bin's shared table (own cluster included)
// to the vertex's gtab region in the layout of tab_cap, and leaves the hubs'
// global tables in place.  The next pass applies the previous pass's moves
// to those tables in place (Algorithm 2's update of the affected tables: a
// mover from X to Y takes w(u, v) from S(u, X) and adds it to S(u, Y) for
// each neighbour u that keeps a table), then reads the argmax of those
// vertices from their tables; vertices of lower degree aggregate from the
// CSR as in every other pass.  Keys are never removed: a sum that reaches
// 0 marks a cluster no longer adjacent and is skipped.  A table that runs
// out of slots is listed and rebuilt from the labels.

// Subtracts w from the sum of an existing key (nothing is inserted).
// Returns false when the key is absent, which only an overflowed table
// (rebuilt afterwards) can show.  Keys present before the kernel come
// before any empty slot of their probe sequence, so concurrent inserts of
// other keys cannot hide them.
__device__ __forceinline__ bool tab_sub(unsigned long long *t, uint32_t cap, int32_t key, int32_t w) {
  const unsigned long long tag = (unsigned long long)((uint32_t)key + 1u) << 32;
  uint32_t s = slot_of(key, cap);
  for (uint32_t probe = 0; probe < cap; ++probe) {
    const unsigned long long cur = t[s];
    if (cur == kEmptySlot) return false;
    if ((cur & 0xFFFFFFFF00000000ull) == tag) {
      atomicAdd(reinterpret_cast<unsigned int *>(&t[s]), (unsigned int)(-w));
      return true;
    }
    s = (s + 1 == cap) ? 0 : s + 1;
  }
  return false;
}

__device__ __forceinline__ void mark_dirty(const PassArgs &a, int32_t u) {
  if (atomicExch(&a.dirty[u], 1) == 0) a.dirty_list[atomicAdd(&a.sc->tab_dirty, 1)] = u;
}

// The move Xo -> Xn of one mover applied to the kept tables of its
// neighbours over edges [e0, e1) (strided by 32, loads batched U at a time).
__device__ __forceinline__ void tab_move_edges(const PassArgs &a, int64_t e0, int64_t e1, int lane,
                                               int32_t Xo, int32_t Xn) {
  constexpr int U = 4;
  for (int64_t base = e0 + lane; base < e1; base += 32 * U) {
    int32_t u[U], w[U];
    int64_t ub[U], ue[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int64_t e = base + 32 * k;
      u[k] = -1;
      w[k] = 0;
      if (e < e1) {
        u[k] = __ldg(a.g.col + e);
        w[k] = __ldg(a.g.ew + e);
      }
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      ub[k] = u[k] >= 0 ? a.g.rp[u[k]] : 0;
      ue[k] = u[k] >= 0 ? a.g.rp[u[k] + 1] : 0;
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      if (u[k] < 0 || ue[k] - ub[k] <= kTabMinDeg) continue;  // no kept table
      unsigned long long *t = a.gtab + 2 * ub[k];
      const uint32_t cap = tab_cap(ue[k] - ub[k]);
      bool fresh;
      const bool ok = tab_sub(t, cap, Xo, w[k]);
      if (!(table_add(t, cap, Xn, w[k], fresh) && ok)) mark_dirty(a, u[k]);
    }
  }
}

// Update: one warp per chunk of a mover's row (the chunks were listed by
// the last pass's apply step).
__global__ void __launch_bounds__(256) k_tab_update(PassArgs a) {
  const int cnt = a.sc->upd_prev;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  long long done = 0;  // edges applied (lane 0), for the profile's byte count
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < cnt; j += nw) {
    const int2 ch = a.upd_list[j];
    const int32_t v = ch.x;
    const int32_t Xo = a.Cprev[v], Xn = a.C[v];
    if (Xo == Xn) continue;  // a mover that got its own emptied id back
    const int64_t e0 = a.g.rp[v] + (int64_t)ch.y * kUpdChunk;
    const int64_t end = a.g.rp[v + 1];
    const int64_t e1 = e0 + kUpdChunk < end ? e0 + kUpdChunk : end;
    tab_move_edges(a, e0, e1, lane, Xo, Xn);
    if (lane == 0) done += e1 - e0;
  }
  flush_block_sum(done, &a.sc->tab_upd_edges);
}

// Rebuilds the listed overflowed tables from the current labels, one warp
// per table (rare: a table overflows only after more new clusters reached
// it than it has free slots).
__global__ void __launch_bounds__(256) k_tab_rebuild(PassArgs a) {
  const int cnt = a.sc->tab_dirty;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  bool ok = true;
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < cnt; j += nw) {
    const int32_t v = a.dirty_list[j];
    const int64_t beg = a.g.rp[v], deg = a.g.rp[v + 1] - beg;
    unsigned long long *t = a.gtab + 2 * beg;
    const uint32_t cap = tab_cap(deg);
    for (int64_t s = lane; s < 2 * deg; s += 32) t[s] = kEmptySlot;
    __syncwarp();
    for (int64_t e = beg + lane; e < beg + deg; e += 32) {
      bool fresh;
      ok &= table_add(t, cap, LC_IDX(a.C[LC_IDX(__ldg(a.g.col + e), a.g.n, kDbgColumn)], a.g.n, kDbgLabel),
                      __ldg(a.g.ew + e), fresh);
    }
    __syncwarp();
    if (lane == 0) a.dirty[v] = 0;
  }
  if (!ok) {
    a.sc->error = 1;
    LC_DBG_FAIL(kDbgProbe, -1, a.g.n);  // the table of one of this thread's listed vertices
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && cnt > 0) a.sc->tab_rebuilt += cnt;
}

// Best (gain, cluster) over the slot pairs [p0, p1) of a kept table
// (16-byte loads, strided by GS, V pairs per thread at a time) and this
// thread's part of S(v, C[v]); with `reset` the slots are cleared as they
// are read (the last pass of a call leaves gtab clean).
template <int GS, int V>
__device__ __forceinline__ void tab_pairs_scan(const PassArgs &a, const GraphParam &P, ulonglong2 *t2,
                                               uint32_t p0, uint32_t p1, int32_t Cv, long long wv,
                                               bool reset, long long &self, long long &gb, int32_t &xb) {
  const long long Lam = P.Lam, muw = P.mu * wv;
  for (uint32_t base = p0 + threadIdx.x; base < p1; base += GS * V) {
    unsigned long long t[2 * V];
    long long WX[2 * V];
    bool use[2 * V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const uint32_t p = base + k * GS;
      ulonglong2 x = make_ulonglong2(kEmptySlot, kEmptySlot);
      if (p < p1) x = t2[p];
      if (reset && p < p1 && (x.x | x.y) != 0ull) t2[p] = make_ulonglong2(kEmptySlot, kEmptySlot);
      t[2 * k] = x.x;
      t[2 * k + 1] = x.y;
    }
#pragma unroll
    for (int k = 0; k < 2 * V; ++k) {
      const int32_t X = slot_key(t[k]), S = slot_val(t[k]);
      use[k] = t[k] != kEmptySlot && S > 0 && X != Cv;
      if (t[k] != kEmptySlot && X == Cv) self += S;
      WX[k] = use[k] ? a.W[X] : 0;
    }
#pragma unroll
    for (int k = 0; k < 2 * V; ++k) {
      if (!use[k]) continue;
      const int32_t X = slot_key(t[k]);
      const long long g = Lam * (long long)slot_val(t[k]) - muw * WX[k];
      if (better(g, X, gb, xb)) {
        gb = g;
        xb = X;
      }
    }
  }
}

// Argmax and candidate test of Algorithm 2 from the kept tables, one block
// per vertex of bins 5-8 (a single reduction to thread 0 per vertex; the
// partials alternate between two buffers, so one barrier per vertex).
template <int GS, int V>
__global__ void __launch_bounds__(GS) k_tab_scan(PassArgs a, const int32_t *__restrict__ list,
                                                 int64_t count) {
  __shared__ long long rs[2][GS / 32], rg[2][GS / 32];
  __shared__ int32_t rx[2][GS / 32];
  long long cntL = 0, phi = 0;
  int par = 0;
  for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
    const int32_t v = list[i];
    const int64_t beg = a.g.rp[v];
    const uint32_t cap = tab_cap(a.g.rp[v + 1] - beg);
    const int32_t Cv = a.C[v];
    const long long wv = a.g.vw[v];
    const GraphParam P = a.gp[graph_of(a, v)];
    long long self = 0, gb = LLONG_MIN;
    int32_t xb = kNone;
    tab_pairs_scan<GS, V>(a, P, reinterpret_cast<ulonglong2 *>(a.gtab + 2 * beg), 0, cap / 2, Cv, wv,
                          a.tab_reset != 0, self, gb, xb);
    group_argmax<32>(gb, xb);
    self = warp_sum(self);
    if ((threadIdx.x & 31) == 0) {
      rg[par][threadIdx.x >> 5] = gb;
      rx[par][threadIdx.x >> 5] = xb;
      rs[par][threadIdx.x >> 5] = self;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < GS / 32; ++w) {
        self += rs[par][w];
        if (better(rg[par][w], rx[par][w], gb, xb)) {
          gb = rg[par][w];
          xb = rx[par][w];
        }
      }
      const long long gC = gain_self(P, self, wv, a.W[Cv]);
      add_self(a, v, gC, phi);
      decide(a, P, v, gC, xb, gb, cntL);
    }
    par ^= 1;
  }
  flush_block_sum(cntL, &a.sc->count_L);
  flush_block_sum(phi, &a.phi_acc[0]);
}

// Hubs: each chunk scans its share of the hub's table; k_hub_decide
// combines the partials and the parts of S(v, C[v]).
__global__ void __launch_bounds__(kHubThreads) k_hub_tab_scan(PassArgs a) {
  const int c = blockIdx.x;
  const int h = a.hub.hub_of[c];
  const int32_t v = a.hub.vtx[h];
  const int64_t beg = a.g.rp[v];
  const GraphParam P = a.gp[graph_of(a, v)];
  long long self = 0, gb = LLONG_MIN;
  int32_t xb = kNone;
  // a chunk of edges [e0, e1) owns the slot pairs [e0 - beg, e1 - beg)
  tab_pairs_scan<kHubThreads, 4>(a, P, reinterpret_cast<ulonglong2 *>(a.gtab + 2 * beg),
                                 (uint32_t)(a.hub.e0[c] - beg), (uint32_t)(a.hub.e1[c] - beg), a.C[v],
                                 a.g.vw[v], a.tab_reset != 0, self, gb, xb);
  hub_part_store(a, c, gb, xb);
  hub_acc_add(a, h, self);
}

// ----------------------------------------------------------- update

// Apply D for M (Algorithm 2, Update): real destinations move now; movers
// to a new empty cluster leave their cluster and are flagged for ids.
__global__ void k_apply(PassArgs a, uint8_t *__restrict__ E) {
  long long empties = 0;
  const int lane = threadIdx.x & 31;
  // warp-uniform trip count: the lists below are appended per warp
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.g.n;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = base + threadIdx.x;
    int nch = 0;         // chunks of this mover's row for the kept tables' update
    bool listed = false;  // a mover for the final objective's update
    if (v < a.g.n) {
      uint8_t e = 0;
      if (a.M[v]) {
        const int32_t Dv = a.D[v], Cv = a.C[v];
        const long long wv = a.g.vw[v];
        a.Cprev[v] = Cv;
        if (a.upd_list || a.movers) {
          const int64_t deg = a.g.rp[v + 1] - a.g.rp[v];
          if (a.upd_list) nch = (int)((deg + kUpdChunk - 1) / kUpdChunk);
          listed = a.movers && deg <= a.hub_min;  // hubs: k_hub_delta_in
        }
        atomicAdd((unsigned long long *)&a.W[Cv], (unsigned long long)(-wv));
        if (Dv >= 0) {
          a.C[v] = LC_IDX(Dv, a.g.n, kDbgDest);
          atomicAdd((unsigned long long *)&a.W[LC_IDX(Dv, a.g.n, kDbgDest)], (unsigned long long)wv);
        } else {
          e = 1;
          empties++;
        }
      }
      E[v] = e;
    }
    if (a.upd_list) {  // uniform over the launch
      int incl = nch;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
      }
      const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
      int first = 0;
      if (lane == 31 && total > 0) first = atomicAdd(&a.sc->upd_count, total);
      first = __shfl_sync(0xFFFFFFFFu, first, 31) + incl - nch;
      for (int c = 0; c < nch; ++c) a.upd_list[first + c] = make_int2((int32_t)v, c);
    }
    if (a.movers) {  // uniform over the launch
      const unsigned m = __ballot_sync(0xFFFFFFFFu, listed);
      int first = 0;
      if (lane == 0 && m) first = atomicAdd(&a.sc->n_movers, __popc(m));
      first = __shfl_sync(0xFFFFFFFFu, first, 0);
      if (listed) a.movers[first + __popc(m & ((1u << lane) - 1u))] = (int32_t)v;
    }
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
// Per graph, the ids left unused after every other move go, ascending, to
// that graph's empty-cluster movers in ascending vertex order.  Labels of a
// graph stay inside its own vertex range, so the free ids of graph g and its
// movers are both ranked from the graph's first vertex vbase:
//   freepos[x] = free ids before x, freelist = all free ids in order,
//   mrank[v]   = movers before v,
//   mover v of graph g gets freelist[freepos[vbase] + mrank[v] - mrank[vbase]].
struct FreeFlag {
  const int32_t *used;
  __device__ int32_t operator()(int64_t x) const { return used[x] == 0 ? 1 : 0; }
};
struct FreeEmit {
  int32_t *freelist, *freepos;
  __device__ void operator()(int64_t x, int32_t pos, int32_t f) const {
    freepos[x] = pos;
    if (f) freelist[pos] = (int32_t)x;
  }
};
struct MoverFlag {
  const uint8_t *E;
  __device__ int32_t operator()(int64_t v) const { return E[v]; }
};
struct MoverEmit {
  int32_t *mrank;
  __device__ void operator()(int64_t v, int32_t pos, int32_t) const { mrank[v] = pos; }
};

__global__ void k_assign_free(PassArgs a, const uint8_t *__restrict__ E,
                              const int32_t *__restrict__ freelist, const int32_t *__restrict__ freepos,
                              const int32_t *__restrict__ mrank) {
  if (a.sc->empty_movers == 0) return;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.g.n;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (!E[v]) continue;
    const int g = graph_of(a, (int32_t)v);
    const int32_t vb = a.gp[g].vbase;
    const int64_t idx = (int64_t)freepos[vb] + mrank[v] - mrank[vb];
    const int32_t x = (idx >= 0 && idx < a.g.n) ? freelist[idx] : -1;
    // there are always at least as many free ids in a graph as movers; an
    // id outside the graph would be a bound violation, reported, not used
    if (x < 0 || x >= a.g.n || graph_of(a, x) != g) {
      a.sc->error = 1;
      continue;
    }
    a.C[v] = x;
    a.W[x] = a.g.vw[v];
  }
}

// Per-graph objective of a batch: sums the recorded g(v, C[v]) by graph.
// Lanes of a warp with the same graph are combined before the atomic.
__global__ void k_graph_sums(PassArgs a) {
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.g.n;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = base + threadIdx.x;
    const bool on = v < a.g.n;
    const int g = on ? graph_of(a, (int32_t)v) : -1;
    long long x = on ? a.gself[v] : 0;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, g);
    const int leader = __ffs(peers) - 1;
    // sum over peers: each lane adds its value into the leader's slot
    __shared__ long long part[1024];
    part[threadIdx.x] = 0;
    __syncwarp();
    if (on) atomicAdd((unsigned long long *)&part[(threadIdx.x & ~31) + leader], (unsigned long long)x);
    __syncwarp();
    if (on && (threadIdx.x & 31) == leader && part[threadIdx.x] != 0)
      atomicAdd((unsigned long long *)&a.phi_acc[g], (unsigned long long)part[threadIdx.x]);
    __syncwarp();
  }
}

// ----------------------------------------------------------- best-of

__global__ void k_pass_begin(Scalars *sc, int advance) {
  if (advance) {
    const int i = sc->pass_idx++;
    sc->phi_live[0] = sc->phi_tab[i & 15][0];
    sc->phi_live[1] = sc->phi_tab[i & 15][1];
  }
  for (int g = 0; g < kAbGroups; ++g) sc->ab_count[g] = 0;
  sc->count_L = 0;
  sc->count_M = 0;
  sc->empty_movers = 0;
  sc->tab_dirty = 0;
  sc->n_movers = 0;
  sc->upd_prev = sc->upd_count;
  sc->upd_count = 0;
}

// Algorithm 2's best-of test, per graph, on the objective accumulated in
// phi_acc (strict improvement keeps the earliest maximum).
__global__ void k_bestof_test(long long *phi_acc, long long *phi_out, int *improved, int G) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    const long long p = phi_acc[g];
    if (p > phi_out[g]) {
      phi_out[g] = p;
      improved[g] = 1;
    } else {
      improved[g] = 0;
    }
    phi_acc[g] = 0;
  }
}

__global__ void k_bestof_copy(PassArgs a, int32_t *__restrict__ C_out) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.g.n;
       v += (int64_t)gridDim.x * blockDim.x)
    if (a.improved[graph_of(a, (int32_t)v)]) C_out[v] = a.C[v];
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

__global__ void k_hub_rows(const int64_t *__restrict__ rp, const int32_t *__restrict__ vtx, int H,
                           int64_t *__restrict__ out) {
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < H; h += gridDim.x * blockDim.x) {
    out[2 * h] = rp[vtx[h]];
    out[2 * h + 1] = rp[vtx[h] + 1];
  }
}

// ================================================================ host

static inline unsigned blocks_for(int64_t items, int per_block) {
  int64_t b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (unsigned)b;
}

// table (8 bytes per slot) + claimed-slot list (2 bytes per half slot)
static constexpr int block_table_bytes(int slots) { return slots * 8; }

void configure_kernels() {
  cudaFuncSetAttribute(k_move_block<64, 1024, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       block_table_bytes(1024));
  cudaFuncSetAttribute(k_move_block<128, 2048, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       block_table_bytes(2048));
  cudaFuncSetAttribute(k_move_block<256, 4096, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       block_table_bytes(4096));
  cudaFuncSetAttribute(k_move_block<256, 6144, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       block_table_bytes(6144));
  cudaFuncSetAttribute(k_move_block<64, 1024, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       block_table_bytes(1024));
  cudaFuncSetAttribute(k_move_block<128, 2048, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       block_table_bytes(2048));
  cudaFuncSetAttribute(k_move_block<256, 4096, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       block_table_bytes(4096));
  cudaFuncSetAttribute(k_move_block<256, 6144, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       block_table_bytes(6144));
}

void build_bins(const LevelGraph &g, const BinPlan &plan, Bins &b, int32_t *scan_tmp, cudaStream_t s) {
  cudaMemsetAsync(b.offs, 0, sizeof(int32_t), s);
  int64_t lo = -1;
  for (int k = 0; k < kBins; ++k) {
    const int64_t hi = k < kBins - 1 ? plan.max_deg[k] : INT64_MAX;
    scan_apply<int32_t>(g.n, BinFlag{g.rp, lo, hi}, BinEmit{b.lists, b.offs + k}, scan_tmp, s);
    k_bin_next_offset<<<1, 1, 0, s>>>(b.offs, k, scan_tmp + scan_tiles(g.n));
    lo = hi;
  }
}

void finish_bins(Bins &b, const int32_t *h_offs) {
  for (int k = 0; k < kBins; ++k) {
    b.list[k] = b.lists + h_offs[k];
    b.rec[k] = b.recs + h_offs[k];
    b.count[k] = h_offs[k + 1] - h_offs[k];
  }
}

__global__ void k_vertex_records(LevelGraph g, const int32_t *__restrict__ gid, const int32_t *__restrict__ lists,
                                 VRec *__restrict__ recs) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = lists[i];
    VRec r;
    r.v = v;
    r.beg = g.rp[v];
    r.deg = (int32_t)(g.rp[v + 1] - r.beg);
    r.g = gid ? gid[v] : 0;
    r.pad = 0;
    r.w = g.vw[v];
    recs[i] = r;
  }
}

void launch_vertex_records(const LevelGraph &g, const int32_t *gid, Bins &b, cudaStream_t s) {
  if (g.n > 0) k_vertex_records<<<blocks_for(g.n, 256), 256, 0, s>>>(g, gid, b.lists, b.recs);
}

void launch_hub_rows(const int64_t *rp, const int32_t *vtx, int H, int64_t *out, cudaStream_t s) {
  if (H > 0) k_hub_rows<<<blocks_for(H, 256), 256, 0, s>>>(rp, vtx, H, out);
}

template <int GS>
static int launch_vertex_kernel(void (*k)(PassArgs, const VRec *, int64_t), const PassArgs &a,
                                BinRange r, cudaStream_t s, size_t smem = 0) {
  if (r.count <= 0) return 0;
  const int threads = GS > 32 ? GS : 256;
  const int per_block = GS > 32 ? 1 : threads / GS;
  k<<<blocks_for(r.count, per_block), threads, smem, s>>>(a, r.rec, r.count);
  return 1;
}

// The same over the plain vertex list (kernels that need little of a record).
template <int GS>
static int launch_list_kernel(void (*k)(PassArgs, const int32_t *, int64_t), const PassArgs &a, BinRange r,
                              cudaStream_t s) {
  if (r.count <= 0) return 0;
  const int threads = GS > 32 ? GS : 256;
  const int per_block = GS > 32 ? 1 : threads / GS;
  k<<<blocks_for(r.count, per_block), threads, 0, s>>>(a, r.list, r.count);
  return 1;
}

static inline unsigned hub_final_blocks(int H) { return blocks_for(H, 256); }

// Kernels without tables take runs of bins: bin 0 -> 1 thread, 1 -> 16
// lanes, 2..4 -> one warp, 5..6 -> 128 threads, 7..8 -> 512 threads.
int launch_first_pass(const PassArgs &a, const Bins &b, cudaStream_t s) {
  int n = 0;
  n += launch_vertex_kernel<1>(k_first_pass<1>, a, bin_range(b, 0, 0), s);
  n += launch_vertex_kernel<16>(k_first_pass<16>, a, bin_range(b, 1, 1), s);
  n += launch_vertex_kernel<32>(k_first_pass<32>, a, bin_range(b, 2, 4), s);
  n += launch_vertex_kernel<128>(k_first_pass<128>, a, bin_range(b, 5, 6), s);
  n += launch_vertex_kernel<512>(k_first_pass<512>, a, bin_range(b, 7, 8), s);
  if (a.hub.H > 0) {
    k_hub_first<<<a.hub.Q, kHubThreads, 0, s>>>(a);
    k_hub_decide<<<hub_final_blocks(a.hub.H), 256, 0, s>>>(a, 1);
    n += 2;
  }
  return n;
}

template <int GS, int SLOTS>
static int launch_move_block(const PassArgs &a, BinRange r, cudaStream_t s) {
  if (r.count <= 0) return 0;
  if (a.tab_build)
    k_move_block<GS, SLOTS, true><<<blocks_for(r.count, 1), GS, block_table_bytes(SLOTS), s>>>(a, r.rec,
                                                                                               r.count);
  else
    k_move_block<GS, SLOTS, false><<<blocks_for(r.count, 1), GS, block_table_bytes(SLOTS), s>>>(a, r.rec,
                                                                                                r.count);
  return 1;
}

template <int SLOTS>
static int launch_move_warp(const PassArgs &a, BinRange r, cudaStream_t s) {
  if (r.count <= 0) return 0;
  k_move_warp<SLOTS><<<blocks_for(r.count, kWarpBinWarps), kWarpBinWarps * 32, 0, s>>>(a, r.rec, r.count);
  return 1;
}

// Bins 0-4 (degree <= 256): aggregation from the CSR in every pass.
static int launch_move_low(const PassArgs &a, const Bins &b, cudaStream_t s) {
  int n = 0;
  const BinRange r0 = bin_range(b, 0, 0);
  if (r0.count > 0) {
    k_move_thread<<<blocks_for(r0.count, 256), 256, 0, s>>>(a, r0.rec, r0.count);
    n++;
  }
  n += launch_vertex_kernel<16>(k_move_small<16>, a, bin_range(b, 1, 1), s);
  n += launch_vertex_kernel<32>(k_move_small<32>, a, bin_range(b, 2, 2), s);
  n += launch_move_warp<256>(a, bin_range(b, 3, 3), s);
  n += launch_move_warp<512>(a, bin_range(b, 4, 4), s);
  return n;
}

int launch_move(const PassArgs &a, const Bins &b, cudaStream_t s) {
  int n = launch_move_low(a, b, s);
  n += launch_move_block<64, 1024>(a, bin_range(b, 5, 5), s);
  n += launch_move_block<128, 2048>(a, bin_range(b, 6, 6), s);
  n += launch_move_block<256, 4096>(a, bin_range(b, 7, 7), s);
  n += launch_move_block<256, 6144>(a, bin_range(b, 8, 8), s);
  if (a.hub.H > 0) {
    k_hub_move_insert<<<a.hub.Q, kHubThreads, 0, s>>>(a);
    k_hub_move_scan<<<a.hub.Q, kHubThreads, 0, s>>>(a);
    k_hub_decide<<<hub_final_blocks(a.hub.H), 256, 0, s>>>(a, 0);
    n += 3;
  }
  return n;
}

template <int GS, int V>
static int launch_tab_scan(const PassArgs &a, BinRange r, cudaStream_t s) {
  if (r.count <= 0) return 0;
  k_tab_scan<GS, V><<<blocks_for(r.count, 1), GS, 0, s>>>(a, r.list, r.count);
  return 1;
}

int launch_table_pass(const PassArgs &a, const Bins &b, cudaStream_t s) {
  int n = launch_move_low(a, b, s);
  k_tab_update<<<152 * 8, 256, 0, s>>>(a);
  k_tab_rebuild<<<152 * 4, 256, 0, s>>>(a);
  n += 2;
  // one 16-byte pair of slots per thread per batch of V: bin 5 has at most
  // 512 pairs, bin 6 1024, bin 7 2048, bin 8 3072
  n += launch_tab_scan<128, 4>(a, bin_range(b, 5, 5), s);
  n += launch_tab_scan<256, 4>(a, bin_range(b, 6, 6), s);
  n += launch_tab_scan<512, 4>(a, bin_range(b, 7, 8), s);
  if (a.hub.H > 0) {
    k_hub_tab_scan<<<a.hub.Q, kHubThreads, 0, s>>>(a);
    k_hub_decide<<<hub_final_blocks(a.hub.H), 256, 0, s>>>(a, 0);
    n += 2;
  }
  return n;
}

// One afterburner group: its kernel over the candidates k_ab_prep listed
// (grid sized for the whole group; surplus blocks find no work).
template <int GS>
static int launch_ab_group(const PassArgs &a, const Bins &b, int g, cudaStream_t s) {
  const BinRange r = bin_range(b, kAbFirstBin[g], kAbFirstBin[g + 1] - 1);
  if (r.count <= 0) return 0;
  const int threads = GS > 32 ? GS : 256;
  const int per_block = GS > 32 ? 1 : threads / GS;
  k_afterburner<GS><<<blocks_for(r.count, per_block), threads, 0, s>>>(a, a.ab_list + a.ab_off[g],
                                                                        &a.sc->ab_count[g]);
  return 1;
}

void set_ab_groups(PassArgs &a, const Bins &b, const BinPlan &plan) {
  for (int g = 0; g < kAbGroups; ++g) {
    a.ab_off[g] = b.list[kAbFirstBin[g]] - b.list[0];
    a.ab_max[g] = plan.max_deg[kAbFirstBin[g + 1] - 1];
    a.ab_gs[g] = plan.ab_gs[g];
  }
}

// Groups 2-4: 32, 128 or 512 threads per candidate (BinPlan::ab_gs).
static int launch_ab_wide_group(const PassArgs &a, const Bins &b, int g, cudaStream_t s) {
  if (a.ab_gs[g] == 16) return launch_ab_group<16>(a, b, g, s);  // group 2 only
  if (a.ab_gs[g] == 32) return launch_ab_group<32>(a, b, g, s);
  if (a.ab_gs[g] == 128) return launch_ab_group<128>(a, b, g, s);
  return launch_ab_group<512>(a, b, g, s);
}

int launch_afterburner(const PassArgs &a, const Bins &b, cudaStream_t s) {
  int n = 1;
  k_ab_prep<<<blocks_for(a.g.n, 256), 256, 0, s>>>(a);
  n += launch_ab_group<1>(a, b, 0, s);
  n += launch_ab_group<16>(a, b, 1, s);
  for (int g = 2; g < kAbGroups; ++g) n += launch_ab_wide_group(a, b, g, s);
  if (a.hub.H > 0) {
    k_hub_afterburner<<<a.hub.Q, kHubThreads, 0, s>>>(a);
    k_hub_ab_final<<<hub_final_blocks(a.hub.H), 256, 0, s>>>(a);
    n += 2;
  }
  return n;
}

// ------------------------------------- symmetry-breaking ablations

__global__ void k_cluster_sizes(const int32_t *__restrict__ C, int32_t *__restrict__ size, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&size[C[v]], 1);
}

// M[v] for every candidate, except (mlh) a vertex alone in its cluster
// whose destination is another one-vertex cluster with a larger label.
__global__ void k_symmetry_ablation(PassArgs a, const int32_t *__restrict__ size, int mlh) {
  long long cntM = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.g.n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t Dv = a.D[v], Cv = a.C[v];
    bool keep = Dv != kNone;
    if (keep && mlh && size[Cv] == 1 && Dv >= 0 && size[Dv] == 1 && Dv > Cv) keep = false;
    a.M[v] = keep;
    cntM += keep;
  }
  flush_block_sum(cntM, &a.sc->count_M);
}

int launch_symmetry_ablation(const PassArgs &a, bool mlh, int32_t *size, cudaStream_t s) {
  if (a.g.n == 0) return 0;
  int n = 1;
  if (mlh) {
    cudaMemsetAsync(size, 0, sizeof(int32_t) * (size_t)a.g.n, s);
    k_cluster_sizes<<<blocks_for(a.g.n, 256), 256, 0, s>>>(a.C, size, a.g.n);
    n++;
  }
  k_symmetry_ablation<<<blocks_for(a.g.n, 256), 256, 0, s>>>(a, size, mlh ? 1 : 0);
  return n;
}

int launch_objective(const PassArgs &a, const Bins &b, cudaStream_t s) {
  int n = 0;
  n += launch_list_kernel<1>(k_objective<1>, a, bin_range(b, 0, 0), s);
  n += launch_list_kernel<16>(k_objective<16>, a, bin_range(b, 1, 1), s);
  n += launch_list_kernel<32>(k_objective<32>, a, bin_range(b, 2, 4), s);
  n += launch_list_kernel<128>(k_objective<128>, a, bin_range(b, 5, 6), s);
  n += launch_list_kernel<512>(k_objective<512>, a, bin_range(b, 7, 8), s);
  if (a.hub.H > 0) {
    k_hub_objective<<<a.hub.Q, kHubThreads, 0, s>>>(a);
    k_hub_obj_final<<<hub_final_blocks(a.hub.H), 256, 0, s>>>(a);
    n += 2;
  }
  return n;
}

// ------------------------- objective after the last pass (one graph)
//
// Phi = Lam IN - mu Q (Eq. 1 regrouped): IN = sum_v S(v, C[v]) and
// Q = sum_X W(X)^2 - sum_v w(v)^2.  The last pass's move step sums Phi of
// the state entering it; its moves change IN only on the movers' edges, by
// ([C'[v] = C'[u]] - [C[v] = C[u]]) w(u, v) per direction, and Q follows
// from W before and after (an O(n) sweep each).  So the objective of the
// call's final state, which the best-of test of Algorithm 2 needs, costs a
// walk over the movers' rows instead of a sweep of the whole graph:
//   Phi' = Phi + Lam dIN - mu (Q' - Q).

// Change of IN over edges [e0, e1) of mover v (strided by GS): an edge to
// a non-mover counts both directions, an edge between movers one (the
// other mover counts the other).
template <int GS>
__device__ __forceinline__ long long delta_in_edges(const PassArgs &a, int32_t v, int64_t e0, int64_t e1,
                                                    int r) {
  constexpr int U = 4;
  const int32_t Cvn = a.C[v], Cvo = a.Cprev[v];
  long long d = 0;
  for (int64_t base = e0 + r; base < e1; base += (int64_t)GS * U) {
    int32_t u[U], w[U], Cun[U];
    uint8_t mu[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int64_t e = base + (int64_t)k * GS;
      u[k] = -1;
      w[k] = 0;
      if (e < e1) {
        u[k] = LC_IDX(__ldg(a.g.col + e), a.g.n, kDbgColumn);
        w[k] = __ldg(a.g.ew + e);
      }
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      Cun[k] = u[k] >= 0 ? a.C[u[k]] : 0;
      mu[k] = u[k] >= 0 ? a.M[u[k]] : 0;
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      if (u[k] < 0) continue;
      const int32_t Cuo = mu[k] ? a.Cprev[u[k]] : Cun[k];
      const int s = (Cvn == Cun[k] ? 1 : 0) - (Cvo == Cuo ? 1 : 0);
      d += (long long)(mu[k] ? 1 : 2) * s * w[k];
    }
  }
  return d;
}

// The per-graph accumulators of the objective update: a.obj holds
// [Phi entering | Q entering | Q after | dIN], G entries each.
__device__ __forceinline__ long long *obj_phi_enter(const PassArgs &a) { return a.obj; }
__device__ __forceinline__ long long *obj_q_enter(const PassArgs &a) { return a.obj + a.G; }
__device__ __forceinline__ long long *obj_q_final(const PassArgs &a) { return a.obj + 2 * a.G; }
__device__ __forceinline__ long long *obj_d_in(const PassArgs &a) { return a.obj + 3 * a.G; }

// dIN over the listed movers (not hubs), one warp each; a batch (BATCH)
// adds each mover's change to its own graph's sum.
template <bool BATCH>
__global__ void __launch_bounds__(256) k_delta_in(PassArgs a) {
  const int cnt = a.sc->n_movers;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  long long d = 0, edges = 0;
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < cnt; j += nw) {
    const int32_t v = a.movers[j];
    const int64_t beg = a.g.rp[v], end = a.g.rp[v + 1];
    const long long dv = delta_in_edges<32>(a, v, beg, end, lane);
    if constexpr (BATCH) {
      const long long t = warp_sum(dv);
      if (lane == 0 && t != 0) atomicAdd((unsigned long long *)&obj_d_in(a)[a.gid[v]], (unsigned long long)t);
    } else {
      d += dv;
    }
    if (lane == 0) edges += end - beg;
  }
  if (!BATCH) flush_block_sum(d, obj_d_in(a));
  flush_block_sum(edges, &a.sc->dphi_edges);
}

__global__ void __launch_bounds__(kHubThreads) k_hub_delta_in(PassArgs a) {
  __shared__ long long rs[kHubThreads / 32];
  const int c = blockIdx.x;
  const int32_t v = a.hub.vtx[a.hub.hub_of[c]];
  if (!a.M[v]) return;  // block-uniform
  const long long d =
      Grp<kHubThreads>::sum(delta_in_edges<kHubThreads>(a, v, a.hub.e0[c], a.hub.e1[c], threadIdx.x), rs);
  if (threadIdx.x == 0) {
    if (d != 0) atomicAdd((unsigned long long *)&obj_d_in(a)[graph_of(a, v)], (unsigned long long)d);
    atomicAdd((unsigned long long *)&a.sc->dphi_edges, (unsigned long long)(a.hub.e1[c] - a.hub.e0[c]));
  }
}

// Q = sum_x W(x)^2 - w(x)^2 over the level's ids x (W of an unused id is 0)
// into q[0] (zeroed by the caller).  Unsigned arithmetic: exact whenever Q
// fits (mu > 0 and the guard Lam T + mu V^2 < 2^60); with mu = 0 it is not
// used.
__global__ void k_q(PassArgs a, long long *q) {
  long long t = 0;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < a.g.n;
       x += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long W = (unsigned long long)a.W[x], w = (unsigned long long)a.g.vw[x];
    t += (long long)(W * W - w * w);
  }
  flush_block_sum(t, q);
}

// The same per graph of a batch, into q[g].  The labels of a graph lie in
// its own vertex range, so the lanes of a warp cover a few runs of one graph
// each; each run is summed by a segmented shuffle scan and added once.
__global__ void k_q_batch(PassArgs a, long long *q) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.g.n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = base + threadIdx.x;
    long long t = 0;
    if (x < a.g.n) {
      const unsigned long long W = (unsigned long long)a.W[x], w = (unsigned long long)a.g.vw[x];
      t = (long long)(W * W - w * w);
    }
    const int g = x < a.g.n ? a.gid[x] : -1;
    // inclusive scan within runs of equal g
    const int gp = __shfl_up_sync(0xFFFFFFFFu, g, 1);
    const bool head = lane == 0 || gp != g;
    unsigned heads = __ballot_sync(0xFFFFFFFFu, head);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xFFFFFFFFu, t, o);
      // lanes o back are in the same run if no head lies in (lane - o, lane]
      const unsigned span = (lane >= o) ? (((1u << lane) << 1) - (1u << (lane - o + 1))) : 0u;
      if (lane >= o && (heads & span) == 0) t += y;
    }
    const int gn = __shfl_down_sync(0xFFFFFFFFu, g, 1);
    const bool tail = lane == 31 || gn != g;
    if (tail && g >= 0 && t != 0) atomicAdd((unsigned long long *)&q[g], (unsigned long long)t);
  }
}

static void launch_q(const PassArgs &a, long long *q, cudaStream_t s) {
  if (a.gid)
    k_q_batch<<<blocks_for(a.g.n, 256), 256, 0, s>>>(a, q);
  else
    k_q<<<blocks_for(a.g.n, 256), 256, 0, s>>>(a, q);
}

__global__ void k_save_phi_enter(PassArgs a) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.G; g += gridDim.x * blockDim.x)
    obj_phi_enter(a)[g] = a.phi_acc[g];
}

__global__ void k_final_phi(PassArgs a) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.G; g += gridDim.x * blockDim.x) {
    const GraphParam P = a.gp[g];
    const long long dq = obj_q_final(a)[g] - obj_q_enter(a)[g];
    a.phi_acc[g] = obj_phi_enter(a)[g] + P.Lam * obj_d_in(a)[g] - (P.mu != 0 ? P.mu * dq : 0);
  }
}

int launch_last_pass_enter(const PassArgs &a, cudaStream_t s) {
  cudaMemsetAsync(a.obj + a.G, 0, sizeof(long long) * (size_t)a.G, s);
  if (a.g.n > 0) launch_q(a, a.obj + a.G, s);
  return a.g.n > 0 ? 1 : 0;
}

int launch_save_phi_enter(const PassArgs &a, cudaStream_t s) {
  k_save_phi_enter<<<blocks_for(a.G, 256), 256, 0, s>>>(a);
  return 1;
}

int launch_final_objective(const PassArgs &a, cudaStream_t s) {
  cudaMemsetAsync(a.obj + 2 * a.G, 0, 2 * sizeof(long long) * (size_t)a.G, s);  // Q after, dIN
  if (a.gid)
    k_delta_in<true><<<152 * 8, 256, 0, s>>>(a);
  else
    k_delta_in<false><<<152 * 8, 256, 0, s>>>(a);
  int n = 1;
  if (a.hub.H > 0) {
    k_hub_delta_in<<<a.hub.Q, kHubThreads, 0, s>>>(a);
    n++;
  }
  if (a.g.n > 0) {
    launch_q(a, a.obj + 2 * a.G, s);
    n++;
  }
  k_final_phi<<<blocks_for(a.G, 256), 256, 0, s>>>(a);
  return n + 1;
}

int launch_apply(const PassArgs &a, const ApplyScratch &w, cudaStream_t s) {
  k_apply<<<blocks_for(a.g.n, 256), 256, 0, s>>>(a, w.E);
  const int *k = &a.sc->empty_movers;
  k_zero_if<<<blocks_for(a.g.n, 256), 256, 0, s>>>(w.used, a.g.n, k);
  k_mark_occupied<<<blocks_for(a.g.n, 256), 256, 0, s>>>(a.C, w.E, w.used, a.g.n, k);
  scan_apply<int32_t>(a.g.n, FreeFlag{w.used}, FreeEmit{w.freelist, w.freepos}, w.scan_tmp, s, k);
  scan_apply<int32_t>(a.g.n, MoverFlag{w.E}, MoverEmit{w.mrank}, w.scan_tmp, s, k);
  k_assign_free<<<blocks_for(a.g.n, 256), 256, 0, s>>>(a, w.E, w.freelist, w.freepos, w.mrank);
  return 10;
}

void launch_pass_begin(Scalars *sc, cudaStream_t s, int advance) { k_pass_begin<<<1, 1, 0, s>>>(sc, advance); }

int launch_graph_sums(const PassArgs &a, cudaStream_t s) {
  if (!a.gself) return 0;
  k_graph_sums<<<blocks_for(a.g.n, 256), 256, 0, s>>>(a);
  return 1;
}

// phi_final[g] = phi_out[g] for the graphs that ran in this call.
__global__ void k_keep_phi(const GraphParam *gp, const long long *phi_out, long long *phi_final, int G) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x)
    if (gp[g].active) phi_final[g] = phi_out[g];
}

int launch_keep_phi(const PassArgs &a, long long *phi_final, cudaStream_t s) {
  k_keep_phi<<<blocks_for(a.G, 256), 256, 0, s>>>(a.gp, a.phi_out, phi_final, a.G);
  return 1;
}

int launch_bestof(const PassArgs &a, int32_t *C_out, cudaStream_t s) {
  k_bestof_test<<<blocks_for(a.G, 256), 256, 0, s>>>(a.phi_acc, a.phi_out, a.improved, a.G);
  k_bestof_copy<<<blocks_for(a.g.n, 256), 256, 0, s>>>(a, C_out);
  return 2;
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
