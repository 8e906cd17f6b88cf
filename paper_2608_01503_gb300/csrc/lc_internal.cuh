// lc_internal.cuh — internal types and device helpers of liblc (sm_103a).
//
// Notation follows Section II of the paper: lambda = mu / Lam, w(v) vertex
// weights, w(u,v) edge weights, S(v,X) = sum of w(u,v) over neighbours u of v
// in cluster X, W(X) = sum of w(u) over u in X.  Gains are Lam-scaled so they
// are exact int64:  g(v,X) = Lam*S(v,X) - mu*w(v)*(W(X) - [X = C[v]] w(v)).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lc.h"
#include "lc_debug.cuh"

namespace lc {

constexpr int32_t kNone = -1;   // D[v]: v is not a candidate
constexpr int32_t kEmpty = -2;  // D[v]: move v to a new empty cluster
// Hash slot = [key + 1 : 32 | value : 32]; 0 is an empty slot, so a table is
// cleared with a plain memset.
constexpr unsigned long long kEmptySlot = 0ull;
constexpr int kMaxLevels = 256;

// Degree bins of the per-vertex kernels.  By default (the boundaries are
// runtime parameters, see BinPlan) a vertex of degree d is handled by
//   bin 0: d <= 8       one thread (aggregation in registers)
//   bin 1: d <= 16      16 lanes, one neighbour per lane (2 vertices per warp)
//   bin 2: d <= 32      one warp, one neighbour per lane
//   bin 3: d <= 128     one warp, shared table of 256 slots
//   bin 4: d <= 256     one warp, shared table of 512 slots
//   bin 5: d <= 512     64 threads, shared table of 1024 slots
//   bin 6: d <= 1024    128 threads, shared table of 2048 slots
//   bin 7: d <= 2048    256 threads, shared table of 4096 slots
//   bin 8: d <= 4096    256 threads, shared table of 6144 slots (load <= 2/3)
//   bin 9: d >  4096    "hubs": the row is cut into chunks of 2048 edges
//                       processed by independent blocks, aggregation in the
//                       vertex's region of the global table (2d slots), then
//                       one finalize step per hub
// A vertex's table holds 2d slots at most, so the shared memory a bin
// reserves per vertex tracks its degree and many vertices stay in flight.
// Kernels without tables launch once over a contiguous range of bins.
constexpr int kBins = 10;
constexpr int kHubBin = kBins - 1;
// The largest degree each bin's kernel can take (its registers or shared
// table), which is also the default bin boundary.
constexpr int64_t kBinMaxDeg[kBins - 1] = {8, 16, 32, 128, 256, 512, 1024, 2048, 4096};
constexpr int kWarpBinWarps = 8;    // warps per block in the warp-table bins
constexpr int kHubThreads = 256;
constexpr int kHubChunk = 2048;     // edges per hub chunk (default)
constexpr int kBin8Slots = 6144;    // shared table of bin 8
constexpr int64_t kTabMinDeg = 256; // kept tables (opts.tables): vertices of degree above this
constexpr int kUpdChunk = 256;      // edges per chunk of a mover's row in the table update

// Degree bins of one call (lc_opts.bin_max_deg / hub_chunk): bin k takes
// max_deg[k-1] < deg <= max_deg[k] (bin 0 from degree 0), the hub bin the
// rows above max_deg[kBins - 2], in chunks of hub_chunk edges.  Every
// max_deg[k] <= kBinMaxDeg[k], so each vertex fits its kernel.
struct BinPlan {
  int64_t max_deg[kBins - 1];
  int64_t hub_chunk;
  int32_t ab_gs[5];  // threads per candidate of each afterburner group
  int64_t hub_min() const { return max_deg[kBins - 2]; }  // hubs: deg > hub_min()
};
inline BinPlan default_bin_plan() {
  BinPlan p;
  for (int k = 0; k < kBins - 1; ++k) p.max_deg[k] = kBinMaxDeg[k];
  p.hub_chunk = kHubChunk;
  const int32_t gs[5] = {1, 16, 32, 128, 512};
  for (int k = 0; k < 5; ++k) p.ab_gs[k] = gs[k];
  return p;
}
// The kept tables' layout depends on the bins above degree 256 only.
inline bool is_default_plan(const BinPlan &p) {
  for (int k = 0; k < kBins - 1; ++k)
    if (p.max_deg[k] != kBinMaxDeg[k]) return false;
  return p.hub_chunk == kHubChunk;
}

// Slots of the kept table of a vertex of degree d, in shared memory and in
// its region gtab[2 rp[v], 2 rp[v+1]) of the global table alike: 2d (load at
// most 1/2), except bin 8, whose shared table holds 6144 slots (load <= 2/3).
// One layout in both places lets a pass copy a shared table out verbatim
// and later passes update it in place.
__host__ __device__ __forceinline__ uint32_t tab_cap(int64_t deg) {
  return (uint32_t)((deg > 2048 && deg <= 4096) ? (2 * deg < kBin8Slots ? 2 * deg : kBin8Slots)
                                                 : 2 * deg);
}

// One level's graph G_l (device pointers).
struct LevelGraph {
  int64_t n, nnz;
  const int64_t *rp;
  const int32_t *col;
  const int32_t *ew;
  const int64_t *vw;
};

// Hub chunks of one level (bin 6).  Chunk c covers edges [e0[c], e1[c]) of
// hub hub_of[c]; the chunks of hub h are [c0[h], c0[h+1]).
struct Hubs {
  int32_t H = 0, Q = 0;
  const int32_t *vtx = nullptr;     // [H] hub vertex ids
  const int32_t *hub_of = nullptr;  // [Q]
  const int64_t *e0 = nullptr, *e1 = nullptr;  // [Q]
  const int32_t *c0 = nullptr;      // [H+1]
  long long *acc = nullptr;         // [H] per-hub sums, zero between uses
  long long *part_g = nullptr;      // [Q] per-chunk argmax partials
  int32_t *part_x = nullptr;        // [Q]
};

// Per-graph constants of a (packed) batch: lambda = mu / Lam, the first
// vertex of the graph in the current level's packed vertex range, and
// whether the graph runs local-move passes at this level.
struct GraphParam {
  long long mu, Lam;
  int32_t vbase;
  int32_t active;
};

// Call-wide constants of the afterburner order (Section IV-A-1).
struct Method {
  int32_t eps_num, eps_den;
  uint32_t seed;
};

// A vertex of a level as the per-vertex kernels need it, stored in bin order
// beside the bin lists once per level: its id, degree, graph and row start,
// and w(v), so that a kernel reads its vertex in one coalesced 32-byte load
// instead of a chain of gathers through the list entry.
struct __align__(16) VRec {
  int32_t v, deg, g, pad;
  int64_t beg;
  long long w;
};

// Afterburner record of a vertex for one pass: its cluster, destination and
// priority bucket packed into one 16-byte load.
struct __align__(16) AbRec {
  int32_t C, D;
  long long q;
};

// Everything the afterburner needs about one listed candidate v itself, written
// by the record pass beside its list entry so that the group kernels read it
// in one coalesced 64-byte load instead of a chain of gathers: its id,
// cluster, destination, degree, hash and graph base, ordering bucket,
// mu w(v), Lambda, row start and delta_v.
struct __align__(16) AbWork {
  int32_t v, C, D, deg;
  uint32_t hv;
  int32_t vbase;
  long long q, muw, Lam, beg, delta;
};

// Device-resident counters of one call (all graphs of a batch together).
struct Scalars {
  int empty_movers;      // movers to a new empty cluster in this pass
  long long count_L, count_M;
  int error;             // internal bound violation (hash probe overrun)
  int pad;
  long long cand_edges;  // stored edges of all candidates, summed over the call's passes
  long long tab_upd_edges; // kept tables: movers' edges applied in place, summed over the call
  int tab_dirty;         // kept tables that overflowed in this pass's update (listed)
  int upd_count;         // chunks of movers' rows listed by this pass's apply step
  int upd_prev;          // ... by the last pass's (read by this pass's table update)
  int pad2;
  long long tab_rebuilt; // kept tables rebuilt, summed over the call's passes
  long long dphi_edges;  // movers' edges read for the objective update, summed over the call
  int n_movers;          // entries of PassArgs::movers
  int pad3;
  long long distinct_x;  // (vertex, adjacent cluster) pairs whose W(X) the move step read,
                         // summed over the call (the argmax's gathers, for the profile)
  // candidates listed per afterburner group in this pass: per-warp atomics
  // of the record pass, on a line of their own
  alignas(128) int ab_count[8];
  // device-side temperature schedule (graph replays): k_pass_begin loads
  // phi_live from phi_tab[pass_idx] and advances pass_idx
  int pass_idx;
  int phi_live[2];
  int pad5;
  int phi_tab[16][2];
};

// The afterburner's launches group the degree bins (one kernel each):
// bin 0, bin 1, bins 2-4, bins 5-6, bins 7-8; hubs go by chunks.
constexpr int kAbGroups = 5;
constexpr int kAbFirstBin[kAbGroups + 1] = {0, 1, 2, 5, 7, 9};

// ------------------------------------------------------------------ hashes

// MurmurHash3 32-bit finaliser (Appleby), a published bijective mixer.
__host__ __device__ inline uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

// Slot of a cluster id in a table of `cap` slots (multiplicative hash then
// Lemire's multiply-shift range reduction; cap need not be a power of two).
__device__ __forceinline__ uint32_t slot_of(int32_t key, uint32_t cap) {
  uint32_t h = (uint32_t)key * 0x9E3779B1u;
  return (uint32_t)(((uint64_t)h * cap) >> 32);
}

__device__ __forceinline__ int32_t slot_key(unsigned long long s) {
  return (int32_t)((uint32_t)(s >> 32) - 1u);
}
__device__ __forceinline__ int32_t slot_val(unsigned long long s) { return (int32_t)(uint32_t)s; }

// Insert (key, w) into an open-addressing table of `cap` 64-bit slots with
// linear probing.  A new key is claimed and its first weight stored in one
// compare-and-swap; later weights of the key are one 32-bit atomic add on
// the value word (values stay below 2^31, so it never reaches the key).
// Returns false when all `cap` slots were probed without success, a bound
// violation (every caller sizes tables to at least twice its distinct keys).
// When this call claimed a new slot, `fresh` is set and `slot` names it.
__device__ __forceinline__ bool table_add(unsigned long long *tab, uint32_t cap, int32_t key,
                                          int32_t w, bool &fresh, uint32_t &slot) {
  const unsigned long long tag = (unsigned long long)((uint32_t)key + 1u) << 32;
  uint32_t s = slot_of(key, cap);
  for (uint32_t probe = 0; probe < cap; ++probe) {
    unsigned long long cur = tab[s];
    if (cur == kEmptySlot) {
      unsigned long long prev = atomicCAS(&tab[s], kEmptySlot, tag | (uint32_t)w);
      if (prev == kEmptySlot) {
        fresh = true;
        slot = s;
        return true;
      }
      cur = prev;
    }
    if ((cur & 0xFFFFFFFF00000000ull) == tag) {
      // value word = low 32 bits of the little-endian slot
      atomicAdd(reinterpret_cast<unsigned int *>(&tab[s]), (unsigned int)w);
      return true;
    }
    s = (s + 1 == cap) ? 0 : s + 1;
  }
  return false;
}

__device__ __forceinline__ bool table_add(unsigned long long *tab, uint32_t cap, int32_t key,
                                          int32_t w, bool &fresh) {
  uint32_t slot;
  return table_add(tab, cap, key, w, fresh, slot);
}

// --------------------------------------------------------------- gains

// Lam-scaled gain of joining cluster X (X != C[v]): Lam*S - mu*w(v)*W(X).
__device__ __forceinline__ long long gain_other(const GraphParam &p, long long S, long long wv,
                                                long long WX) {
  return p.Lam * S - p.mu * wv * WX;
}
// Lam-scaled gain of staying: Lam*S_self - mu*w(v)*(W(C[v]) - w(v)).
__device__ __forceinline__ long long gain_self(const GraphParam &p, long long S, long long wv,
                                               long long WC) {
  return p.Lam * S - p.mu * wv * (WC - wv);
}

// Better (gain, id) for the argmax: larger gain, ties to the smaller id.
__device__ __forceinline__ bool better(long long g1, int32_t x1, long long g2, int32_t x2) {
  return g1 > g2 || (g1 == g2 && (uint32_t)x1 < (uint32_t)x2);
}

// floor(eps_den * delta / (eps_num * Lam)), the epsilon bucket of the
// ordering of Section IV-A-1 (eps_num, eps_den, Lam > 0).  The products are
// formed in 128 bits; when both fit in 64 bits, as they do unless delta or
// Lam is near the exactness guards, one 64-bit division replaces the far
// costlier 128-bit one.  Either way the quotient is exact.
__device__ __forceinline__ long long eps_bucket(const Method &m, long long Lam, long long delta) {
  const __int128 num = (__int128)m.eps_den * delta;
  const __int128 den = (__int128)m.eps_num * Lam;
  if (num == (__int128)(long long)num && den == (__int128)(long long)den) {
    const long long n64 = (long long)num, d64 = (long long)den;
    long long q = n64 / d64;  // truncates toward zero
    if (q * d64 != n64 && n64 < 0) q -= 1;
    return q;
  }
  __int128 qq = num / den;
  if (qq * den != num && num < 0) qq -= 1;
  return (long long)qq;
}

// ord(u) < ord(v): larger bucket first, then smaller hash, then smaller id.
__device__ __forceinline__ bool earlier(long long qu, uint32_t hu, int32_t u, long long qv,
                                        uint32_t hv, int32_t v) {
  if (qu != qv) return qu > qv;
  if (hu != hv) return hu < hv;
  return u < v;
}

// --------------------------------------------------------- reductions

template <typename T>
__device__ __forceinline__ T warp_sum(T x, unsigned mask = 0xFFFFFFFFu) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o);
  return x;
}

// Sum within aligned groups of G lanes (G a power of two <= 32).
template <int G, typename T>
__device__ __forceinline__ T group_sum(T x) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
  return x;
}

// Argmax (gain, id) within aligned groups of G lanes.
template <int G>
__device__ __forceinline__ void group_argmax(long long &g, int32_t &x) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    long long g2 = __shfl_xor_sync(0xFFFFFFFFu, g, o);
    int32_t x2 = __shfl_xor_sync(0xFFFFFFFFu, x, o);
    if (better(g2, x2, g, x)) {
      g = g2;
      x = x2;
    }
  }
}

// ------------------------------------------------------------- launch

inline int grid_for(int64_t work, int per_block, int cap = 152 * 32) {
  int64_t b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

}  // namespace lc
