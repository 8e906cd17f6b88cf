// lc_leiden.cuh — launch interface of lc_leiden.cu (pLeiden, Section V).
#pragma once

#include "lc_internal.cuh"

namespace lc {

// SplitMix64's output function (Steele, Lea and Flood, 2014) on a counter:
// value number c of the stream (seed, level, stream).
__host__ __device__ inline uint64_t sm64_mix(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}
__host__ __device__ inline uint64_t stream_rand(uint32_t seed, int32_t level, int32_t stream,
                                                int64_t c) {
  const uint64_t key =
      sm64_mix(((uint64_t)seed << 32) ^ ((uint64_t)(uint32_t)level << 8) ^ (uint64_t)(uint32_t)stream);
  return sm64_mix(key + (uint64_t)(c + 1) * 0x9E3779B97F4A7C15ull);
}

// Per-vertex records gathered once per edge by pLeidenR's row sweeps.
struct __align__(16) RefRec {  // constraint label, membership of U, w(v)
  int32_t B;
  int32_t inU;
  long long w;
};
struct __align__(16) KeyRec {  // tree root and ordering key
  int32_t root;
  int32_t pad;
  uint64_t f;
};

// Scratch of LocalMoveAlt and pLeidenR (n = vertices of the level).
struct LeidenScratch {
  int32_t *list;        // [n] non-node-optimal vertices / sort values
  int32_t *list2;       // [n] sort values (ping-pong)
  int32_t *to;          // [n] label taken by each move of LocalMoveAlt
  int32_t *size;        // [n] cluster sizes
  int32_t *H;           // [n] chosen edge (target vertex; v itself = none)
  int32_t *root;        // [n]
  int32_t *first_bad;   // [n] first failing position of each tree (indexed by root)
  int64_t *pos;         // [n] position of each vertex in tree order
  uint64_t *f;          // [n] ordering key
  uint64_t *key;        // [n] sort keys
  uint64_t *key2;       // [n] sort keys (ping-pong)
  int64_t *WB;          // [n] weight of each constraint cluster
  int64_t *SB;          // [n] S(v, B[v])
  int64_t *Sv;          // [n] weight to earlier vertices of the tree
  int64_t *tv;          // [n] the vertex's term of w(C, B minus C) along the tree order
  int64_t *ps_w;        // [n] exclusive prefix of w over the tree order
  int64_t *ps_t;        // [n] exclusive prefix of the external-weight terms
  uint8_t *flags;       // [n + 4] bit 0: in U, 1: kept edge, 2: has a kept child, 3: key fixed
  int64_t *scan64;      // scan scratch: scan_scratch(max(n, radix_hist_len(n)))
  int32_t *hist;        // radix histograms: radix_hist_len(n)
  int64_t *scal;        // [4] device scalars: m, committed, error
  RefRec *rec;          // [n]
  KeyRec *krec;         // [n]
};

// Elements of hist / scan64 the radix sort of n keys needs.
int64_t radix_hist_len(int64_t n);

// LocalMoveAlt (Section V-A) on labels C (in place), given D and delta of a
// pass with phi = 0 (D = kNone: no move with gD >= gC).  W: cluster weights
// of C (modified).  Leaves the number of committed moves in scal[1].
void launch_local_move_alt(const LevelGraph &g, const GraphParam *gp, int32_t *C, const int32_t *D,
                           const int64_t *delta, int64_t *W, LeidenScratch &ls, int *error,
                           cudaStream_t s);
// pLeidenR (Algorithm 6) with constraint B (dense labels in [0, n)): refined
// labels R (tree root ids, or the vertex itself).  bins: the level's degree
// bins (per-vertex kernels use a thread up to degree 32, a warp above).
struct Bins;
void launch_pleiden_refine(const LevelGraph &g, const Bins &bins, const GraphParam *gp, const int32_t *B,
                           uint32_t seed, int32_t level, int32_t *R, LeidenScratch &ls, int *error,
                           cudaStream_t s);
// Downsample: Cc[Cd[v]] = C[v] for every v (Cc: int32[n_c]).
void launch_downsample(const int32_t *Cd, const int32_t *C, int32_t *Cc, int64_t n, cudaStream_t s);

}  // namespace lc
