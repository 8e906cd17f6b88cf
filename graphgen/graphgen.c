/*
 * graphgen.c — seeded synthetic graph generators and the CSR builder.
 *
 * Input infrastructure only: these routines build the undirected, weighted
 * graphs that both the CPU oracle and the CUDA path consume.  Nothing here
 * computes any part of the clustering method (no gains, no objective, no
 * contraction).  The output is a symmetric CSR with both directions of every
 * undirected edge stored, rows sorted by column, no self-loops, no duplicate
 * edges and strictly positive integer weights (the graph model of Section II:
 * positive integer vertex and edge weights, w(u,v)=0 iff (u,v) is not an edge).
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * SplitMix64 (Steele, Lea & Flood, 2014), both written from their published
 * definitions.  Edge weights are a stateless SplitMix64 mix of the canonical
 * endpoint pair, so w(u,v) = w(v,u) by construction and does not depend on
 * generation order.
 *
 * Families:
 *   gg_sbm    planted-partition stochastic block model, per-block-pair
 *             Bernoulli edges drawn by geometric skipping (Batagelj & Brandes,
 *             "Efficient generation of large random networks", 2005).
 *   gg_rmat   R-MAT (Chakrabarti, Zhan & Faloutsos, 2004) with the Graph500
 *             quadrant probabilities, no noise, no vertex permutation;
 *             symmetrised, deduplicated, self-loops removed.
 *   gg_grid3d 3-D 7-point-stencil lattice (6 neighbours, no wraparound) with a
 *             fraction of edges rewired: the higher endpoint is replaced by a
 *             uniform vertex (loops re-drawn, duplicates removed).
 *   gg_from_edges  CSR builder from an arbitrary undirected edge list.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int64_t n, nnz;
  int64_t *row_ptr; /* n+1 */
  int32_t *col;     /* nnz */
  int32_t *ew;      /* nnz */
} gg_csr;

enum { GG_OK = 0, GG_ERR_ARG = 1, GG_ERR_OOM = 2 };

/* ---------------------------------------------------------------- PRNG --- */

static uint64_t splitmix64_step(uint64_t *state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Stateless mixer: SplitMix64 output function applied to one input word. */
static uint64_t mix64(uint64_t x) {
  uint64_t s = x;
  return splitmix64_step(&s);
}

typedef struct {
  uint64_t s[4];
} xoshiro;

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t xo_next(xoshiro *r) {
  uint64_t *s = r->s;
  const uint64_t out = rotl64(s[1] * 5, 7) * 9;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return out;
}

static void xo_seed(xoshiro *r, uint64_t seed) {
  uint64_t st = seed;
  for (int i = 0; i < 4; i++) r->s[i] = splitmix64_step(&st);
}

/* uniform double in (0, 1] */
static double xo_open01(xoshiro *r) { return ((double)(xo_next(r) >> 11) + 1.0) * 0x1.0p-53; }

/* uniform integer in [0, m) for m >= 1 (Lemire's multiply-shift; bias < m/2^64) */
static uint64_t xo_below(xoshiro *r, uint64_t m) {
  return (uint64_t)(((unsigned __int128)xo_next(r) * m) >> 64);
}

/* ------------------------------------------------------------ edge list --- */

typedef struct {
  uint64_t *k; /* canonical key (min << 32) | max */
  int64_t len, cap;
} edgevec;

static int ev_push(edgevec *e, uint64_t key) {
  if (e->len == e->cap) {
    int64_t nc = e->cap ? e->cap * 2 : 1024;
    uint64_t *nk = (uint64_t *)realloc(e->k, (size_t)nc * sizeof(uint64_t));
    if (!nk) return GG_ERR_OOM;
    e->k = nk;
    e->cap = nc;
  }
  e->k[e->len++] = key;
  return GG_OK;
}

static inline uint64_t canon(int64_t u, int64_t v) {
  return u < v ? (((uint64_t)u << 32) | (uint64_t)v) : (((uint64_t)v << 32) | (uint64_t)u);
}

/* LSD radix sort of 64-bit keys, 16-bit digits, only over the digits in use. */
static int radix_sort_u64(uint64_t *a, int64_t len) {
  if (len < 2) return GG_OK;
  uint64_t maxk = 0;
  for (int64_t i = 0; i < len; i++)
    if (a[i] > maxk) maxk = a[i];
  uint64_t *tmp = (uint64_t *)malloc((size_t)len * sizeof(uint64_t));
  if (!tmp) return GG_ERR_OOM;
  int64_t *cnt = (int64_t *)malloc(65536 * sizeof(int64_t));
  if (!cnt) {
    free(tmp);
    return GG_ERR_OOM;
  }
  uint64_t *src = a, *dst = tmp;
  for (int shift = 0; shift < 64 && (maxk >> shift) != 0; shift += 16) {
    memset(cnt, 0, 65536 * sizeof(int64_t));
    for (int64_t i = 0; i < len; i++) cnt[(src[i] >> shift) & 0xFFFF]++;
    int64_t run = 0;
    for (int d = 0; d < 65536; d++) {
      int64_t c = cnt[d];
      cnt[d] = run;
      run += c;
    }
    for (int64_t i = 0; i < len; i++) dst[cnt[(src[i] >> shift) & 0xFFFF]++] = src[i];
    uint64_t *t = src;
    src = dst;
    dst = t;
  }
  if (src != a) memcpy(a, src, (size_t)len * sizeof(uint64_t));
  free(tmp);
  free(cnt);
  return GG_OK;
}

static int64_t sort_unique(uint64_t *a, int64_t len, int *err) {
  *err = radix_sort_u64(a, len);
  if (*err) return 0;
  int64_t m = 0;
  for (int64_t i = 0; i < len; i++)
    if (m == 0 || a[i] != a[m - 1]) a[m++] = a[i];
  return m;
}

static int32_t edge_weight(uint64_t key, uint64_t wseed, int32_t wmin, int32_t wmax) {
  if (wmax <= wmin) return wmin;
  uint64_t span = (uint64_t)(wmax - wmin) + 1;
  return wmin + (int32_t)(mix64(key ^ wseed) % span);
}

/* Build the symmetric CSR from sorted, unique, loop-free canonical keys.
 * Row x lists its lower neighbours (ascending) then its upper neighbours
 * (ascending), so every row is sorted by column. */
static int build_csr(int64_t n, const uint64_t *keys, int64_t m, uint64_t wseed, int32_t wmin,
                     int32_t wmax, gg_csr *out) {
  memset(out, 0, sizeof(*out));
  out->n = n;
  out->nnz = 2 * m;
  out->row_ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  out->col = (int32_t *)malloc((size_t)(2 * m > 0 ? 2 * m : 1) * sizeof(int32_t));
  out->ew = (int32_t *)malloc((size_t)(2 * m > 0 ? 2 * m : 1) * sizeof(int32_t));
  int64_t *fill = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!out->row_ptr || !out->col || !out->ew || !fill) {
    free(fill);
    return GG_ERR_OOM;
  }
  for (int64_t i = 0; i < m; i++) {
    out->row_ptr[(keys[i] >> 32) + 1]++;
    out->row_ptr[(keys[i] & 0xFFFFFFFFu) + 1]++;
  }
  for (int64_t x = 0; x < n; x++) out->row_ptr[x + 1] += out->row_ptr[x];
  memcpy(fill, out->row_ptr, ((size_t)n + 1) * sizeof(int64_t));
  /* lower neighbours: edge (u,v), u<v, contributes u to row v */
  for (int64_t i = 0; i < m; i++) {
    int64_t u = (int64_t)(keys[i] >> 32), v = (int64_t)(keys[i] & 0xFFFFFFFFu);
    int32_t w = edge_weight(keys[i], wseed, wmin, wmax);
    int64_t p = fill[v]++;
    out->col[p] = (int32_t)u;
    out->ew[p] = w;
  }
  /* upper neighbours: contributes v to row u */
  for (int64_t i = 0; i < m; i++) {
    int64_t u = (int64_t)(keys[i] >> 32), v = (int64_t)(keys[i] & 0xFFFFFFFFu);
    int32_t w = edge_weight(keys[i], wseed, wmin, wmax);
    int64_t p = fill[u]++;
    out->col[p] = (int32_t)v;
    out->ew[p] = w;
  }
  free(fill);
  return GG_OK;
}

static int finish(int64_t n, edgevec *e, uint64_t seed, int32_t wmin, int32_t wmax, gg_csr *out) {
  int err = GG_OK;
  int64_t m = sort_unique(e->k, e->len, &err);
  if (err) {
    free(e->k);
    return err;
  }
  err = build_csr(n, e->k, m, mix64(seed ^ 0x5157A11EDULL), wmin, wmax, out);
  free(e->k);
  return err;
}

void gg_free(gg_csr *g) {
  if (!g) return;
  free(g->row_ptr);
  free(g->col);
  free(g->ew);
  memset(g, 0, sizeof(*g));
}

/* ------------------------------------------------------------------ SBM --- */

/* Emit Bernoulli(p) pairs of a block pair by geometric skipping.
 * Diagonal block (size s): pairs (a, b) with b < a < s, the triangle walk of
 * Batagelj & Brandes.  Off-diagonal (si x sj): index t -> (t / sj, t % sj). */
static int sbm_block_pair(xoshiro *r, int64_t base_i, int64_t si, int64_t base_j, int64_t sj,
                          int diag, double p, edgevec *e) {
  if (p <= 0.0 || si <= 0 || sj <= 0) return GG_OK;
  int err;
  if (p >= 1.0) {
    if (diag) {
      for (int64_t a = 1; a < si; a++)
        for (int64_t b = 0; b < a; b++)
          if ((err = ev_push(e, canon(base_i + a, base_i + b)))) return err;
    } else {
      for (int64_t a = 0; a < si; a++)
        for (int64_t b = 0; b < sj; b++)
          if ((err = ev_push(e, canon(base_i + a, base_j + b)))) return err;
    }
    return GG_OK;
  }
  const double lq = log1p(-p);
  if (diag) {
    const double tri = (double)si * (double)(si - 1) / 2.0;
    int64_t a = 1, b = -1;
    while (a < si) {
      double skip = floor(log(xo_open01(r)) / lq);
      if (skip >= tri) break;
      b += 1 + (int64_t)skip;
      while (b >= a && a < si) {
        b -= a;
        a++;
      }
      if (a < si && (err = ev_push(e, canon(base_i + a, base_i + b)))) return err;
    }
  } else {
    const int64_t total = si * sj;
    int64_t t = -1;
    for (;;) {
      double skip = floor(log(xo_open01(r)) / lq);
      if (skip >= (double)total) break;
      t += 1 + (int64_t)skip;
      if (t >= total) break;
      if ((err = ev_push(e, canon(base_i + t / sj, base_j + t % sj)))) return err;
    }
  }
  return GG_OK;
}

/* Planted partition: n vertices in nblocks blocks of sizes as equal as
 * possible (the first n % nblocks blocks get one extra vertex); intra-block
 * pairs are edges with probability p_in, inter-block pairs with p_out. */
int gg_sbm(int64_t n, int64_t nblocks, double p_in, double p_out, uint64_t seed, int32_t wmin,
           int32_t wmax, gg_csr *out) {
  if (!out || n < 0 || n > 0x7FFFFFFF || nblocks < 1 || nblocks > (n > 0 ? n : 1) || wmin < 1 ||
      wmax < wmin)
    return GG_ERR_ARG;
  xoshiro r;
  xo_seed(&r, seed);
  edgevec e = {0};
  int64_t *base = (int64_t *)malloc(((size_t)nblocks + 1) * sizeof(int64_t));
  if (!base) return GG_ERR_OOM;
  base[0] = 0;
  for (int64_t b = 0; b < nblocks; b++) base[b + 1] = base[b] + n / nblocks + (b < n % nblocks);
  int err = GG_OK;
  for (int64_t bi = 0; bi < nblocks && !err; bi++)
    for (int64_t bj = bi; bj < nblocks && !err; bj++)
      err = sbm_block_pair(&r, base[bi], base[bi + 1] - base[bi], base[bj], base[bj + 1] - base[bj],
                           bi == bj, bi == bj ? p_in : p_out, &e);
  free(base);
  if (err) {
    free(e.k);
    return err;
  }
  return finish(n, &e, seed, wmin, wmax, out);
}

/* ----------------------------------------------------------------- RMAT --- */

int gg_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed,
            int32_t wmin, int32_t wmax, gg_csr *out) {
  if (!out || scale < 1 || scale > 30 || edge_factor < 0 || a < 0 || b < 0 || c < 0 ||
      a + b + c > 1.0 || wmin < 1 || wmax < wmin)
    return GG_ERR_ARG;
  const int64_t n = (int64_t)1 << scale;
  const int64_t samples = edge_factor * n;
  /* 32-bit quadrant thresholds */
  const uint64_t ta = (uint64_t)(a * 4294967296.0);
  const uint64_t tb = (uint64_t)((a + b) * 4294967296.0);
  const uint64_t tc = (uint64_t)((a + b + c) * 4294967296.0);
  xoshiro r;
  xo_seed(&r, seed);
  edgevec e = {0};
  e.cap = samples > 0 ? samples : 1;
  e.k = (uint64_t *)malloc((size_t)e.cap * sizeof(uint64_t));
  if (!e.k) return GG_ERR_OOM;
  for (int64_t s = 0; s < samples; s++) {
    int64_t u = 0, v = 0;
    uint64_t word = 0;
    for (int lvl = 0; lvl < scale; lvl++) {
      uint64_t x;
      if ((lvl & 1) == 0) {
        word = xo_next(&r);
        x = word & 0xFFFFFFFFu;
      } else {
        x = word >> 32;
      }
      int ub, vb;
      if (x < ta) {
        ub = 0;
        vb = 0;
      } else if (x < tb) {
        ub = 0;
        vb = 1;
      } else if (x < tc) {
        ub = 1;
        vb = 0;
      } else {
        ub = 1;
        vb = 1;
      }
      u = (u << 1) | ub;
      v = (v << 1) | vb;
    }
    if (u != v) e.k[e.len++] = canon(u, v);
  }
  return finish(n, &e, seed, wmin, wmax, out);
}

/* --------------------------------------------------------------- grid3d --- */

int gg_grid3d(int64_t nx, int64_t ny, int64_t nz, double rewire_p, uint64_t seed, int32_t wmin,
              int32_t wmax, gg_csr *out) {
  if (!out || nx < 1 || ny < 1 || nz < 1 || rewire_p < 0 || rewire_p > 1 || wmin < 1 ||
      wmax < wmin)
    return GG_ERR_ARG;
  const int64_t n = nx * ny * nz;
  if (n > 0x7FFFFFFF) return GG_ERR_ARG;
  const uint64_t tp = (uint64_t)(rewire_p * 18446744073709551616.0 > 18446744073709551615.0
                                     ? 18446744073709551615.0
                                     : rewire_p * 18446744073709551616.0);
  xoshiro r;
  xo_seed(&r, seed);
  edgevec e = {0};
  e.cap = 3 * n + 1;
  e.k = (uint64_t *)malloc((size_t)e.cap * sizeof(uint64_t));
  if (!e.k) return GG_ERR_OOM;
  for (int64_t z = 0; z < nz; z++)
    for (int64_t y = 0; y < ny; y++)
      for (int64_t x = 0; x < nx; x++) {
        const int64_t u = x + nx * (y + ny * z);
        int64_t nb[3];
        int cnt = 0;
        if (x + 1 < nx) nb[cnt++] = u + 1;
        if (y + 1 < ny) nb[cnt++] = u + nx;
        if (z + 1 < nz) nb[cnt++] = u + nx * ny;
        for (int i = 0; i < cnt; i++) {
          int64_t v = nb[i];
          if (rewire_p > 0 && xo_next(&r) < tp && n > 1) {
            do {
              v = (int64_t)xo_below(&r, (uint64_t)n);
            } while (v == u);
          }
          e.k[e.len++] = canon(u, v);
        }
      }
  return finish(n, &e, seed, wmin, wmax, out);
}

/* ------------------------------------------------------------ edge list --- */

/* Build a CSR from m undirected edges (src[i], dst[i]); loops are dropped and
 * duplicates merged (the first occurrence's weight rule is the hash rule, so
 * explicit weights are not taken here: use wmin == wmax for unit weights). */
int gg_from_edges(int64_t n, int64_t m, const int64_t *src, const int64_t *dst, uint64_t seed,
                  int32_t wmin, int32_t wmax, gg_csr *out) {
  if (!out || n < 0 || n > 0x7FFFFFFF || m < 0 || wmin < 1 || wmax < wmin) return GG_ERR_ARG;
  edgevec e = {0};
  e.cap = m > 0 ? m : 1;
  e.k = (uint64_t *)malloc((size_t)e.cap * sizeof(uint64_t));
  if (!e.k) return GG_ERR_OOM;
  for (int64_t i = 0; i < m; i++) {
    if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) {
      free(e.k);
      return GG_ERR_ARG;
    }
    if (src[i] != dst[i]) e.k[e.len++] = canon(src[i], dst[i]);
  }
  return finish(n, &e, seed, wmin, wmax, out);
}
