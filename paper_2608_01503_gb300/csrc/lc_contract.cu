// lc_contract.cu — label compaction, gather-free graph contraction
// (Algorithm 4) and projection (Algorithm 1, ProjectCluster).
//
// Contraction works per FINE vertex (no gathering of fine vertices by
// cluster): coarse vertex x owns the region [2 off[x], 2 off[x+1]) of the
// global hash scratch, where off is the exclusive prefix sum of
// bound[x] = sum of deg(v) over v in C_x (an upper bound on x's distinct
// coarse neighbours, so the load factor stays <= 1/2).  Every fine edge
// (v,u) with C[u] != C[v] is inserted into C[v]'s region; the insert that
// claims a new slot also counts a unique coarse edge of x.  The coarse
// offsets are a scan of those counts and the coarse CSR is one stream
// compaction over all regions, which also resets the slots for reuse.
#include <climits>

#include "lc_contract.cuh"
#include "lc_group.cuh"
#include "lc_internal.cuh"
#include "lc_scan.cuh"

namespace lc {

__global__ void k_mark_used(const int32_t *__restrict__ C, int32_t *__restrict__ used, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    used[C[v]] = 1;
}

// Per-graph dense relabelling.  Labels of graph g lie in its vertex range
// [vbase_g, vbase_g + n_g), so one scan over all labels numbers each graph's
// labels in order; the prefix at each graph's first vertex gives its start.
struct UsedIn {
  const int32_t *used;
  const int32_t *gid;
  const uint8_t *keep;  // nullable: only labels of graphs with keep[g]
  __device__ int32_t operator()(int64_t x) const {
    if (!used[x]) return 0;
    if (keep && !keep[gid ? gid[x] : 0]) return 0;
    return 1;
  }
};
struct NewIdOut {
  int32_t *newid;
  const int32_t *gid;       // nullable (one graph)
  const GraphParam *gp;     // per-graph vertex bases
  int32_t *gstart;          // [G]: prefix at each graph's first vertex
  int32_t *gid_next;        // nullable: graph of each new id
  __device__ void operator()(int64_t x, int32_t pos, int32_t f) const {
    newid[x] = pos;
    const int g = gid ? gid[x] : 0;
    if (gp[g].vbase == x) gstart[g] = pos;
    if (f && gid_next) gid_next[pos] = g;
  }
};

// out[v] = newid[C[v]] - base, where base is the start of v's graph when
// `local` is set (labels numbered within each graph); vertices of graphs
// that do not keep their labels get -1.
__global__ void k_relabel(const int32_t *__restrict__ C, const int32_t *__restrict__ newid,
                          int32_t *__restrict__ out, int64_t n, const int32_t *__restrict__ gid,
                          const int32_t *__restrict__ gstart, const uint8_t *__restrict__ keep,
                          int local) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int g = gid ? gid[v] : 0;
    if (keep && !keep[g]) {
      out[v] = -1;
      continue;
    }
    out[v] = newid[C[v]] - (local ? gstart[g] : 0);
  }
}

// bound[C[v]] += deg(v), vw_c[C[v]] += w(v)
__global__ void k_bound(LevelGraph g, const int32_t *__restrict__ Cd, int64_t *bound, int64_t *vw_c) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = Cd[v];
    if (x < 0) continue;  // graph finished coarsening
    const int64_t d = g.rp[v + 1] - g.rp[v];
    if (d) atomicAdd((unsigned long long *)&bound[x], (unsigned long long)d);
    atomicAdd((unsigned long long *)&vw_c[x], (unsigned long long)g.vw[v]);
  }
}

struct I64In {
  const int64_t *a;
  __device__ int64_t operator()(int64_t i) const { return a[i]; }
};
struct I64Out {
  int64_t *o;
  __device__ void operator()(int64_t i, int64_t pos, int64_t) const { o[i] = pos; }
};

struct InsertArgs {
  LevelGraph g;
  const int32_t *Cd;
  const int64_t *off;
  unsigned long long *tab;
  int32_t *cnt;
  int *error;
  int64_t nc;  // coarse vertices
};

// Insert fine edges [e0, e1) of v leaving C[v] into the coarse table of
// x = C[v] (strided by GS, loads batched U at a time); returns the number of
// slots this thread claimed.
template <int GS>
__device__ __forceinline__ int insert_edges(const InsertArgs &a, int32_t x, int64_t e0, int64_t e1,
                                            int r, bool &ok) {
  constexpr int U = 4;
  const int64_t o0 = a.off[x];
  const uint32_t cap = (uint32_t)(2 * (a.off[x + 1] - o0));
  unsigned long long *tab = a.tab + 2 * o0;
  int fresh_n = 0;
  for (int64_t base = e0; base < e1; base += (int64_t)GS * U) {
    int32_t u[U], w[U], y[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int64_t e = base + k * GS + r;
      u[k] = -1;
      w[k] = 0;
      if (e < e1) {
        u[k] = LC_IDX(__ldg(a.g.col + e), a.g.n, kDbgColumn);
        w[k] = __ldg(a.g.ew + e);
      }
    }
#pragma unroll
    for (int k = 0; k < U; ++k) y[k] = u[k] >= 0 ? LC_IDX(a.Cd[u[k]], a.nc, kDbgCoarse) : x;
#pragma unroll
    for (int k = 0; k < U; ++k) {
      if (y[k] == x) continue;
      bool fresh = false;
      ok &= table_add(tab, cap, y[k], w[k], fresh);
      fresh_n += fresh;
    }
  }
  return fresh_n;
}

template <int GS>
__global__ void __launch_bounds__(GS > 32 ? GS : 256)
    k_insert(InsertArgs a, const int32_t *__restrict__ list, int64_t count) {
  const int r = Grp<GS>::rank();
  for_each_vertex<GS>(count, [&](int64_t i, bool active) {
    if (!active) return;
    const int32_t v = list[i];
    const int32_t x = a.Cd[v];
    if (x < 0) return;  // graph finished coarsening
    bool ok = true;
    const int fresh_n = insert_edges<GS>(a, x, a.g.rp[v], a.g.rp[v + 1], r, ok);
    if (!ok) {
      *a.error = 1;
      LC_DBG_FAIL(kDbgProbe, v, a.g.n);
    }
    if (fresh_n) atomicAdd(&a.cnt[x], fresh_n);
  });
}

// Hub rows: one block per chunk of the level's hub plan.
__global__ void __launch_bounds__(kHubThreads) k_insert_hub(InsertArgs a, Hubs hub) {
  const int c = blockIdx.x;
  const int32_t v = hub.vtx[hub.hub_of[c]];
  const int32_t x = a.Cd[v];
  if (x < 0) return;  // graph finished coarsening
  bool ok = true;
  const int fresh_n = insert_edges<kHubThreads>(a, x, hub.e0[c], hub.e1[c], threadIdx.x, ok);
  if (!ok) {
    *a.error = 1;
    LC_DBG_FAIL(kDbgProbe, v, a.g.n);
  }
  if (fresh_n) atomicAdd(&a.cnt[x], fresh_n);
}

struct CntIn {
  const int32_t *cnt;
  __device__ int64_t operator()(int64_t i) const { return cnt[i]; }
};

struct SlotIn {
  const unsigned long long *tab;
  __device__ int32_t operator()(int64_t s) const { return tab[s] != kEmptySlot ? 1 : 0; }
};
struct SlotOut {
  unsigned long long *tab;
  int32_t *col;
  int32_t *ew;
  __device__ void operator()(int64_t s, int32_t pos, int32_t f) const {
    if (f) {
      const unsigned long long t = tab[s];
      col[pos] = slot_key(t);
      ew[pos] = slot_val(t);
      tab[s] = kEmptySlot;
    }
  }
};

// ProjectCluster.  Labels of a graph live in its own vertex range at every
// level, so a coarse label is rebased from the graph's coarse range to its
// fine range (one graph: both bases are 0).  A graph that finished
// coarsening at this level keeps the singleton clustering its last
// local-move call returned.
__global__ void k_project(const int32_t *__restrict__ Cd, const int32_t *__restrict__ Cnext,
                          int32_t *__restrict__ C, int64_t n, const int32_t *__restrict__ gid,
                          const GraphParam *__restrict__ gp_fine,
                          const GraphParam *__restrict__ gp_coarse) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (Cd[v] < 0) {
      C[v] = (int32_t)v;
      continue;
    }
    const int g = gid ? gid[v] : 0;
    C[v] = gp_fine[g].vbase + (Cnext[Cd[v]] - gp_coarse[g].vbase);
  }
}

// gid[v] = the graph whose vertex range [gptr[g], gptr[g+1]) holds v.
__global__ void k_graph_ids(const int64_t *__restrict__ gptr, int G, int32_t *__restrict__ gid, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = G;  // gptr[lo] <= v < gptr[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (gptr[mid] <= v)
        lo = mid;
      else
        hi = mid;
    }
    gid[v] = lo;
  }
}

// ================================================================= host

static inline unsigned blocks_for(int64_t items, int per_block) {
  int64_t b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (unsigned)b;
}

void launch_mark_used(const int32_t *C, int64_t n, int32_t *used, cudaStream_t s) {
  cudaMemsetAsync(used, 0, sizeof(int32_t) * (size_t)(n > 0 ? n : 1), s);
  k_mark_used<<<blocks_for(n, 256), 256, 0, s>>>(C, used, n);
}

void launch_number_labels(const int32_t *used, int64_t n, const int32_t *gid, const GraphParam *gp,
                          const uint8_t *keep, int32_t *newid, int32_t *gstart, int32_t *gid_next,
                          int32_t *scan_tmp, cudaStream_t s) {
  scan_apply<int32_t>(n, UsedIn{used, gid, keep}, NewIdOut{newid, gid, gp, gstart, gid_next}, scan_tmp, s);
}

void launch_relabel(const int32_t *C, const int32_t *newid, int32_t *out, int64_t n, const int32_t *gid,
                    const int32_t *gstart, const uint8_t *keep, int local, cudaStream_t s) {
  k_relabel<<<blocks_for(n, 256), 256, 0, s>>>(C, newid, out, n, gid, gstart, keep, local);
}

const int32_t *compact_total(const int32_t *scan_tmp, int64_t n) {
  return scan_tmp + scan_tiles(n);
}

void launch_contract_offsets(const LevelGraph &g, const int32_t *Cd, int64_t n_c, int64_t *bound,
                             int64_t *off, int64_t *vw_c, int64_t *scan_tmp64, cudaStream_t s) {
  cudaMemsetAsync(bound, 0, sizeof(int64_t) * (size_t)(n_c + 1), s);
  cudaMemsetAsync(vw_c, 0, sizeof(int64_t) * (size_t)(n_c > 0 ? n_c : 1), s);
  k_bound<<<blocks_for(g.n, 256), 256, 0, s>>>(g, Cd, bound, vw_c);
  scan_apply<int64_t>(n_c + 1, I64In{bound}, I64Out{off}, scan_tmp64, s);
}

template <int GS>
static int launch_insert(const InsertArgs &a, const int32_t *list, int64_t count, cudaStream_t s) {
  if (count <= 0) return 0;
  const int threads = GS > 32 ? GS : 256;
  const int per_block = GS > 32 ? 1 : threads / GS;
  k_insert<GS><<<blocks_for(count, per_block), threads, 0, s>>>(a, list, count);
  return 1;
}

int launch_contract_insert(const LevelGraph &g, const int32_t *Cd, const int64_t *off,
                           unsigned long long *tab, int32_t *cnt, int64_t n_c, int *error,
                           const int32_t *const *lists, const int64_t *counts, const Hubs &hub,
                           cudaStream_t s) {
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)(n_c > 0 ? n_c : 1), s);
  InsertArgs a{g, Cd, off, tab, cnt, error, n_c};
  auto range = [&](int lo, int hi) {
    int64_t c = 0;
    for (int k = lo; k <= hi; ++k) c += counts[k];
    return c;
  };
  int n = 0;
  n += launch_insert<1>(a, lists[0], range(0, 0), s);
  n += launch_insert<16>(a, lists[1], range(1, 1), s);
  n += launch_insert<32>(a, lists[2], range(2, 4), s);
  n += launch_insert<128>(a, lists[5], range(5, 6), s);
  n += launch_insert<512>(a, lists[7], range(7, 8), s);
  if (hub.H > 0) {
    k_insert_hub<<<hub.Q, kHubThreads, 0, s>>>(a, hub);
    n++;
  }
  return n;
}

void launch_contract_rowptr(const int32_t *cnt, int64_t n_c, int64_t *rp_c, int64_t *scan_tmp64,
                            cudaStream_t s) {
  scan_apply<int64_t>(n_c, CntIn{cnt}, I64Out{rp_c}, scan_tmp64, s);
  cudaMemcpyAsync(rp_c + n_c, scan_tmp64 + scan_tiles(n_c), sizeof(int64_t),
                  cudaMemcpyDeviceToDevice, s);
}

void launch_contract_compact(unsigned long long *tab, int64_t slots, int32_t *col_c, int32_t *ew_c,
                             int32_t *scan_tmp, cudaStream_t s) {
  scan_apply<int32_t>(slots, SlotIn{tab}, SlotOut{tab, col_c, ew_c}, scan_tmp, s);
}

void launch_graph_ids(const int64_t *gptr, int G, int32_t *gid, int64_t n, cudaStream_t s) {
  k_graph_ids<<<blocks_for(n, 256), 256, 0, s>>>(gptr, G, gid, n);
}

void launch_project(const int32_t *Cd, const int32_t *Cnext, int32_t *C, int64_t n, const int32_t *gid,
                    const GraphParam *gp_fine, const GraphParam *gp_coarse, cudaStream_t s) {
  k_project<<<blocks_for(n, 256), 256, 0, s>>>(Cd, Cnext, C, n, gid, gp_fine, gp_coarse);
}

}  // namespace lc
