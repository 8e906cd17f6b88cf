/*
 * lc_oracle.c — plain, slow, sequential CPU oracle of pLouvain / Louvain+ on
 * the LambdaCC objective.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA path.
 *
 * Notation (Section II): lambda = mu / Lambda (0 <= mu <= Lambda, Lambda > 0),
 * w(v) vertex weights, w(u,v) edge weights, S(v,X) = sum of w(u,v) over
 * neighbours u of v with C[u] = X, W(X) = sum of w(u) over u in X.  All gains
 * are kept Lambda-scaled so they are exact integers:
 *   g(v,X)    = Lambda * w'(v,X)            (Section II-A, w'(X,Y) with X={v})
 *             = Lambda*S(v,X) - mu*w(v)*(W(X) - [X = C[v]] w(v))
 *   g(v,empty) = 0
 *   Phi(C)    = Lambda * lambdaCC(C)        (Eq. 1, ordered pairs u != v)
 * Everything is int64 with int128 where a product can grow.
 *
 * Readings taken where the paper is silent (listed in the design notes):
 *   - argmax over clusters adjacent to v other than C[v]; ties -> smallest id;
 *   - the empty cluster is a fresh label distinct from every other label;
 *   - priority delta_v = g(v,D[v]) - g(v,C[v]) (Algorithm 3's delta, no
 *     factor 2); epsilon buckets q_v = floor(delta_v / (eps * Lambda)), then
 *     hash h_v = fmix32(v xor seed) ascending, then id;
 *   - empty-cluster movers take, in ascending vertex order, the ascending ids
 *     left unused after every other move is applied;
 *   - best-of uses a strict improvement (Algorithm 2, the lambdaCC test).
 *
 * Pins (tests/test_oracle_pins.py): Eq. 1 against the dense pair sum; every
 * gain against objective differences; each pass's destination, empty-cluster
 * rule, candidate test and afterburner value against exhaustive
 * re-evaluation; contraction against a membership-matrix product and the
 * constant objective offset; whole runs against exhaustive search, lambda=0
 * components, networkx modularity and hand-derived closed forms.
 * Algorithm 1's coarsening stop (|C_l| = |V_l|) and the ascending-id label
 * compaction are pinned in tests/test_oracle_coarsening.py by re-running the
 * pinned LocalMovePasses on every traced level and by sparse membership
 * products, with planted early and late stops rejected.
 * Parity unpinned (readings, no passage fixes them): the hash salt and the
 * bucket rounding of the ordering, and which free ids the empty-cluster
 * movers receive; they are pinned only through GPU/oracle bit-exactness.
 *
 * Also here: constrained and iterated Louvain+ (Section V-B), pLeiden and
 * pLeiden+ (Section V: LocalMoveAlt, pLeidenR, Downsample) and the
 * symmetry-breaking ablations of Section VI; their pins are in
 * tests/test_oracle_constrained.py, tests/test_oracle_leiden.py and
 * tests/test_oracle_ablations.py.  Parity unpinned there: the orientation
 * of pLeidenR's kept edges (keys falling towards the root) and the order
 * of LocalMoveAlt's list (ascending ids), which the paper leaves open.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;

/* Built with -fopenmp (the all-core CPU baseline), the loops over vertices
 * inside one synchronous pass and over clusters inside one contraction run
 * on all threads.  Every iteration writes only its own vertex's or
 * cluster's entries, each thread has its own accumulation scratch, and the
 * reductions are integer sums, so the results are identical to the
 * sequential build (which ignores the pragmas). */
#ifdef _OPENMP
static int orc_threads(void) { return omp_get_max_threads(); }
static int orc_thread(void) { return omp_get_thread_num(); }
#else
static int orc_threads(void) { return 1; }
static int orc_thread(void) { return 0; }
#endif

/* ------------------------------------------------------------ types --- */

typedef struct {
  int64_t n, nnz;
  const int64_t *row_ptr; /* n+1 */
  const int32_t *col;     /* nnz */
  const int32_t *ew;      /* nnz, w(u,v) > 0 */
  const int64_t *vw;      /* n,   w(v) >= 0 */
} orc_graph;

typedef struct {
  int64_t lam_num, lam_den; /* lambda = lam_num / lam_den */
  int32_t pass_limit;       /* passes per LocalMovePasses call */
  int32_t phi_num[16], phi_den[16]; /* temperature phi_i of pass i */
  int32_t eps_num, eps_den; /* epsilon of the ordering */
  uint32_t seed;            /* salt of the ordering hash */
  int32_t uncoarsen;        /* 1: Louvain+ (Algorithm 1 line 12), 0: Louvain */
  int32_t symmetry;         /* 0: afterburner filter (Algorithm 3); 1: none, every candidate
                               moves; 2: minimum label heuristic in odd passes, none in even
                               ones (the ablations of Section VI) */
} orc_params;

enum { ORC_EV_PASS = 1, ORC_EV_LMP = 2, ORC_EV_CONTRACT = 3 };
enum { ORC_PHASE_COARSEN = 0, ORC_PHASE_UNCOARSEN = 1 };

/* One trace record, handed to the caller's callback (pointers valid only
 * during the call). */
typedef struct {
  int32_t kind, level, phase, pass; /* pass is 1-based; 0 for non-pass events */
  int64_t n;
  const int32_t *C_before; /* PASS: clustering entering the pass */
  const int32_t *C;        /* PASS: clustering after the pass; LMP: C_out */
  const int32_t *D;        /* PASS: destination; -1 none, -2 empty cluster */
  const uint8_t *in_L;     /* PASS: candidate list membership */
  const uint8_t *in_M;     /* PASS: afterburner survivors */
  const int64_t *delta;    /* PASS: g(v,D[v]) - g(v,C[v]) (0 when D = none) */
  const int64_t *q;        /* PASS: epsilon bucket of delta (valid on L) */
  const int64_t *adj;      /* PASS: afterburner-adjusted delta (valid on L) */
  int64_t phi_hi;          /* PASS: Phi(C) after; LMP: Phi(C_out) */
  uint64_t phi_lo;
  int64_t count_L, count_M;
  /* CONTRACT: the coarse graph G_{level+1} */
  int64_t cn, cnnz;
  const int64_t *c_row_ptr;
  const int32_t *c_col;
  const int32_t *c_ew;
  const int64_t *c_vw;
} orc_event;

typedef void (*orc_callback)(void *ctx, const orc_event *ev);

typedef struct {
  int64_t n_clusters;
  int32_t levels; /* number of graphs G_0..G_top */
  int32_t passes_total;
  int64_t phi_hi;
  uint64_t phi_lo;
  double objective;  /* lambdaCC = Phi / Lambda */
  double modularity; /* (Phi - mu*sum w(v)^2) / (Lambda * sum w(u,v)) */
} orc_result;

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_OOM = 2 };

#define ORC_NONE (-1)
#define ORC_EMPTY (-2)

static void split128(i128 x, int64_t *hi, uint64_t *lo) {
  *hi = (int64_t)(x >> 64);
  *lo = (uint64_t)x;
}

/* --------------------------------------------------- objective (Eq. 1) --- */

/* W(X) for every label X in [0, n). */
static void cluster_weights(const orc_graph *g, const int32_t *C, int64_t *W) {
  memset(W, 0, (size_t)g->n * sizeof(int64_t));
  for (int64_t v = 0; v < g->n; v++) W[C[v]] += g->vw[v];
}

/* Phi(C) = Lambda * lambdaCC(C), Eq. 1 second form:
 *   lambdaCC = sum over ordered pairs (u,v) in env(C) of w(u,v)
 *              - lambda * sum_i sum_{u != v in C_i} w(u) w(v)
 * with sum_{u != v in C_i} w(u) w(v) = W(C_i)^2 - sum_{v in C_i} w(v)^2. */
static i128 objective(const orc_graph *g, int64_t mu, int64_t Lam, const int32_t *C, int64_t *Wscratch) {
  int64_t env = 0; /* at most the sum of all stored weights: nnz < 2^32 entries below 2^31 */
#pragma omp parallel for schedule(static) reduction(+ : env)
  for (int64_t v = 0; v < g->n; v++)
    for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; e++)
      if (C[g->col[e]] == C[v]) env += g->ew[e];
  cluster_weights(g, C, Wscratch);
  i128 pairs = 0;
  for (int64_t x = 0; x < g->n; x++) pairs += (i128)Wscratch[x] * Wscratch[x];
  for (int64_t v = 0; v < g->n; v++) pairs -= (i128)g->vw[v] * g->vw[v];
  return (i128)Lam * env - (i128)mu * pairs;
}

int orc_objective(const orc_graph *g, int64_t mu, int64_t Lam, const int32_t *C, int64_t *phi_hi,
                  uint64_t *phi_lo) {
  if (!g || !C || Lam <= 0) return ORC_ERR_ARG;
  for (int64_t v = 0; v < g->n; v++)
    if (C[v] < 0 || C[v] >= g->n) return ORC_ERR_ARG;
  int64_t *W = (int64_t *)malloc((size_t)(g->n > 0 ? g->n : 1) * sizeof(int64_t));
  if (!W) return ORC_ERR_OOM;
  split128(objective(g, mu, Lam, C, W), phi_hi, phi_lo);
  free(W);
  return ORC_OK;
}

/* g(v, X): Lambda-scaled w'(v, X) under clustering C (Section II-A).
 * X = -2 denotes a new empty cluster (gain 0). */
int orc_gain(const orc_graph *g, int64_t mu, int64_t Lam, const int32_t *C, int64_t v, int32_t X,
             int64_t *out) {
  if (!g || !C || v < 0 || v >= g->n) return ORC_ERR_ARG;
  if (X == ORC_EMPTY) {
    *out = 0;
    return ORC_OK;
  }
  int64_t S = 0, WX = 0;
  for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; e++)
    if (C[g->col[e]] == X) S += g->ew[e];
  for (int64_t u = 0; u < g->n; u++)
    if (C[u] == X) WX += g->vw[u];
  if (X == C[v]) WX -= g->vw[v];
  *out = (int64_t)((i128)Lam * S - (i128)mu * g->vw[v] * WX);
  return ORC_OK;
}

/* ------------------------------------------------------------ ordering --- */

/* MurmurHash3 32-bit finaliser (Appleby), a published bijective mixer. */
static uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

/* floor(a / b) for b > 0 */
static i128 floordiv128(i128 a, i128 b) {
  i128 q = a / b;
  if ((a % b != 0) && (a < 0)) q -= 1;
  return q;
}

/* Section IV-A-1: greater deltas come earlier; deltas in the same epsilon
 * bucket are ordered by the vertex hash, then by id. */
static int earlier(int64_t u, int64_t v, const int64_t *q, uint32_t seed) {
  if (q[u] != q[v]) return q[u] > q[v];
  uint32_t hu = fmix32((uint32_t)u ^ seed), hv = fmix32((uint32_t)v ^ seed);
  if (hu != hv) return hu < hv;
  return u < v;
}

/* --------------------------------------------------------------- pass --- */

typedef struct {
  int64_t n;
  int64_t *W, *acc, *delta, *q, *adj, *gC; /* acc and touched: one n-slice per thread */
  int32_t *touched, *D, *C_before, *C_next, *mark, *Bc;
  uint8_t *in_L, *in_M;
} work;

static void work_free(work *w) {
  free(w->W);
  free(w->acc);
  free(w->delta);
  free(w->q);
  free(w->adj);
  free(w->gC);
  free(w->touched);
  free(w->D);
  free(w->C_before);
  free(w->C_next);
  free(w->mark);
  free(w->Bc);
  free(w->in_L);
  free(w->in_M);
  memset(w, 0, sizeof(*w));
}

static int work_alloc(work *w, int64_t n) {
  memset(w, 0, sizeof(*w));
  size_t m = (size_t)(n > 0 ? n : 1);
  w->n = n;
  w->W = calloc(m, 8);
  const size_t mt = m * (size_t)orc_threads();
  w->acc = calloc(mt, 8);
  w->delta = calloc(m, 8);
  w->q = calloc(m, 8);
  w->adj = calloc(m, 8);
  w->gC = calloc(m, 8);
  w->touched = calloc(mt, 4);
  w->D = calloc(m, 4);
  w->C_before = calloc(m, 4);
  w->C_next = calloc(m, 4);
  w->mark = calloc(m, 4);
  w->Bc = calloc(m, 4);
  w->in_L = calloc(m, 1);
  w->in_M = calloc(m, 1);
  if (!w->W || !w->acc || !w->delta || !w->q || !w->adj || !w->gC || !w->touched || !w->D ||
      !w->C_before || !w->C_next || !w->mark || !w->Bc || !w->in_L || !w->in_M) {
    work_free(w);
    return ORC_ERR_OOM;
  }
  return ORC_OK;
}

#define ORC_MIXED (-1)

/* One synchronous pass of Algorithm 2 (the body of its pass loop) with
 * temperature phi = phi_n / phi_d: destinations and candidate list
 * (Algorithm 2), afterburner filter (Algorithm 3), Update (apply D for M).
 * C is updated in place.
 * With a constraint clustering B (Section V-B, the note on iterating
 * Louvain+; NULL = none), v may only join a cluster X all of whose members
 * u have B[u] = B[v]; Bc[X] holds that common value, ORC_MIXED when the
 * members disagree (such a cluster admits nobody).  Staying and the empty
 * cluster are always allowed. */
static void one_pass(const orc_graph *g, const orc_params *p, const int32_t *B, int32_t pass,
                     int32_t phi_n, int32_t phi_d, int32_t *C, work *w, int64_t *count_L,
                     int64_t *count_M) {
  const int64_t n = g->n, mu = p->lam_num, Lam = p->lam_den;
  memcpy(w->C_before, C, (size_t)n * sizeof(int32_t));
  cluster_weights(g, C, w->W);
  int64_t nL = 0, nM = 0;
  if (B) {
    for (int64_t x = 0; x < n; x++) w->mark[x] = 0; /* mark: Bc[x] is set */
    for (int64_t v = 0; v < n; v++) {
      const int32_t X = C[v];
      if (!w->mark[X]) {
        w->mark[X] = 1;
        w->Bc[X] = B[v];
      } else if (w->Bc[X] != B[v]) {
        w->Bc[X] = ORC_MIXED;
      }
    }
  }

  /* Algorithm 2, parallel loop over V: D[v] = argmax over C \ C[v]. */
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : nL)
  for (int64_t v = 0; v < n; v++) {
    int64_t *acc = w->acc + (int64_t)orc_thread() * n; /* zero between vertices */
    int32_t *touched = w->touched + (int64_t)orc_thread() * n;
    int64_t nt = 0;
    for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; e++) {
      int32_t X = C[g->col[e]];
      if (acc[X] == 0) touched[nt++] = X;
      acc[X] += g->ew[e];
    }
    const int32_t Cv = C[v];
    const int64_t wv = g->vw[v];
    const i128 gC = (i128)Lam * acc[Cv] - (i128)mu * wv * (w->W[Cv] - wv);
    int32_t best = ORC_NONE;
    i128 gbest = 0;
    for (int64_t t = 0; t < nt; t++) {
      const int32_t X = touched[t];
      if (X == Cv) continue;
      if (B && (B[v] == ORC_MIXED || w->Bc[X] != B[v])) continue; /* the constraint forbids X */
      const i128 gX = (i128)Lam * acc[X] - (i128)mu * wv * w->W[X];
      if (best == ORC_NONE || gX > gbest || (gX == gbest && X < best)) {
        best = X;
        gbest = gX;
      }
    }
    for (int64_t t = 0; t < nt; t++) acc[touched[t]] = 0;
    /* empty-cluster rule: both w'(v,C[v]) and w'(v,D[v]) negative */
    if (gC < 0 && (best == ORC_NONE || gbest < 0)) {
      best = ORC_EMPTY;
      gbest = 0;
    }
    /* candidate test: w'(v,D[v]) >= (1 - phi) w'(v,C[v]), times Lambda*phi_d */
    const int inL = best != ORC_NONE && (i128)phi_d * gbest >= (i128)(phi_d - phi_n) * gC;
    w->D[v] = best;
    w->gC[v] = (int64_t)gC;
    w->delta[v] = best == ORC_NONE ? 0 : (int64_t)(gbest - gC);
    w->in_L[v] = (uint8_t)inL;
    w->in_M[v] = 0;
    w->q[v] = 0;
    w->adj[v] = 0;
    nL += inL;
  }

  /* ordering keys of the candidates */
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < n; v++)
    if (w->in_L[v])
      w->q[v] = (int64_t)floordiv128((i128)p->eps_den * w->delta[v], (i128)p->eps_num * Lam);

  if (p->symmetry != 0) {
    /* Ablations: no filter, or the minimum label heuristic (a vertex alone
     * in its cluster may not join another one-vertex cluster with a larger
     * label, so two singletons never swap) in odd passes. */
    const int mlh = p->symmetry == 2 && (pass % 2) == 1;
    int64_t *size = w->acc; /* zero between uses */
    if (mlh)
      for (int64_t v = 0; v < n; v++) size[C[v]]++;
    for (int64_t v = 0; v < n; v++) {
      if (!w->in_L[v]) continue;
      const int32_t Cv = C[v], Dv = w->D[v];
      const int forbid = mlh && size[Cv] == 1 && Dv >= 0 && size[Dv] == 1 && Dv > Cv;
      w->adj[v] = w->delta[v];
      w->in_M[v] = !forbid;
      nM += w->in_M[v];
    }
    if (mlh)
      for (int64_t v = 0; v < n; v++) size[C[v]] = 0;
  }

  /* Algorithm 3: afterburner filter. */
  const int64_t n_ab = p->symmetry == 0 ? n : 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : nM)
  for (int64_t v = 0; v < n_ab; v++) {
    if (!w->in_L[v]) continue;
    i128 d = w->delta[v];
    const int32_t Cv = C[v], Dv = w->D[v];
    for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; e++) {
      const int64_t u = g->col[e];
      if (!w->in_L[u] || !earlier(u, v, w->q, p->seed)) continue;
      const i128 a = (i128)Lam * g->ew[e] - (i128)mu * g->vw[u] * g->vw[v]; /* Lambda w'(u,v) */
      const int32_t Cu = C[u], Du = w->D[u];
      if (Cv == Cu)
        d += a;
      else if (Dv == Cu)
        d -= a;
      if (Cv == Du)
        d -= a;
      else if (Dv >= 0 && Dv == Du)
        d += a;
    }
    w->adj[v] = (int64_t)d;
    w->in_M[v] = d >= 0;
    nM += w->in_M[v];
  }

  /* Update: apply D for M.  Real destinations first; then the empty-cluster
   * movers receive the ids that are unused once every move is applied,
   * ascending ids to ascending vertices. */
  memcpy(w->C_next, C, (size_t)n * sizeof(int32_t));
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < n; v++)
    if (w->in_M[v] && w->D[v] >= 0) w->C_next[v] = w->D[v];
  memset(w->mark, 0, (size_t)n * sizeof(int32_t));
  for (int64_t v = 0; v < n; v++)
    if (!(w->in_M[v] && w->D[v] == ORC_EMPTY)) w->mark[w->C_next[v]] = 1;
  int64_t next_free = 0;
  for (int64_t v = 0; v < n; v++) {
    if (!(w->in_M[v] && w->D[v] == ORC_EMPTY)) continue;
    while (w->mark[next_free]) next_free++; /* a free id exists: used ids < n */
    w->C_next[v] = (int32_t)next_free;
    w->mark[next_free] = 1;
  }
  memcpy(C, w->C_next, (size_t)n * sizeof(int32_t));
  *count_L = nL;
  *count_M = nM;
}

/* ------------------------------------------------- LocalMovePasses --- */

typedef struct {
  orc_callback cb;
  void *ctx;
  int32_t passes_total;
} tracer;

/* Algorithm 2: `limit` synchronous passes from C (in/out); keeps the best
 * lambdaCC clustering seen, including the input (strict improvement). */
static int local_move_passes(const orc_graph *g, const orc_params *p, const int32_t *B, int32_t *C,
                             int level, int phase, tracer *tr, i128 *phi_out_ret) {
  const int64_t n = g->n;
  work w;
  if (work_alloc(&w, n)) return ORC_ERR_OOM;
  int32_t *C_out = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!C_out) {
    work_free(&w);
    return ORC_ERR_OOM;
  }
  memcpy(C_out, C, (size_t)n * sizeof(int32_t));
  i128 phi_out = objective(g, p->lam_num, p->lam_den, C, w.W);
  for (int i = 1; i <= p->pass_limit; i++) {
    int64_t nL = 0, nM = 0;
    one_pass(g, p, B, i, p->phi_num[i - 1], p->phi_den[i - 1], C, &w, &nL, &nM);
    /* one_pass leaves the afterburner arrays intact; W is reused below */
    const i128 phi = objective(g, p->lam_num, p->lam_den, C, w.W);
    if (tr) tr->passes_total++;
    if (tr && tr->cb) {
      orc_event ev;
      memset(&ev, 0, sizeof(ev));
      ev.kind = ORC_EV_PASS;
      ev.level = level;
      ev.phase = phase;
      ev.pass = i;
      ev.n = n;
      ev.C_before = w.C_before;
      ev.C = C;
      ev.D = w.D;
      ev.in_L = w.in_L;
      ev.in_M = w.in_M;
      ev.delta = w.delta;
      ev.q = w.q;
      ev.adj = w.adj;
      split128(phi, &ev.phi_hi, &ev.phi_lo);
      ev.count_L = nL;
      ev.count_M = nM;
      tr->cb(tr->ctx, &ev);
    }
    if (phi > phi_out) {
      phi_out = phi;
      memcpy(C_out, C, (size_t)n * sizeof(int32_t));
    }
  }
  memcpy(C, C_out, (size_t)n * sizeof(int32_t));
  if (tr && tr->cb) {
    orc_event ev;
    memset(&ev, 0, sizeof(ev));
    ev.kind = ORC_EV_LMP;
    ev.level = level;
    ev.phase = phase;
    ev.n = n;
    ev.C = C;
    split128(phi_out, &ev.phi_hi, &ev.phi_lo);
    tr->cb(tr->ctx, &ev);
  }
  if (phi_out_ret) *phi_out_ret = phi_out;
  free(C_out);
  work_free(&w);
  return ORC_OK;
}

static int check_params(const orc_graph *g, const orc_params *p) {
  if (!g || !p || p->symmetry < 0 || p->symmetry > 2) return ORC_ERR_ARG;
  if (g->n < 0 || g->n > 0x7FFFFFFF || p->lam_den <= 0 || p->lam_num < 0 ||
      p->lam_num > p->lam_den || p->pass_limit < 0 || p->pass_limit > 16 || p->eps_num <= 0 ||
      p->eps_den <= 0)
    return ORC_ERR_ARG;
  for (int i = 0; i < p->pass_limit; i++)
    if (p->phi_den[i] <= 0 || p->phi_num[i] < 0 || p->phi_num[i] > p->phi_den[i]) return ORC_ERR_ARG;
  return ORC_OK;
}

/* Public: one LocalMovePasses call from the clustering C (in/out). */
int orc_local_move(const orc_graph *g, const orc_params *p, int32_t *C, orc_callback cb, void *ctx,
                   int64_t *phi_hi, uint64_t *phi_lo) {
  int rc = check_params(g, p);
  if (rc) return rc;
  for (int64_t v = 0; v < g->n; v++)
    if (C[v] < 0 || C[v] >= g->n) return ORC_ERR_ARG;
  tracer tr = {cb, ctx, 0};
  i128 phi = 0;
  rc = local_move_passes(g, p, NULL, C, 0, ORC_PHASE_COARSEN, &tr, &phi);
  if (!rc && phi_hi && phi_lo) split128(phi, phi_hi, phi_lo);
  return rc;
}

/* ------------------------------------------------------- contraction --- */

/* Coarse graph of Section III-A: one coarse vertex x per cluster C_x with
 * weight w(C_x); coarse edges (x,y) and (y,x) with weight w(C_x, C_y) iff
 * that weight is positive; no self-loops (intra-cluster weight is dropped).
 * C must be dense in [0, n_c).  Rows are emitted sorted by column. */
typedef struct {
  int64_t n, nnz;
  int64_t *row_ptr;
  int32_t *col;
  int32_t *ew;
  int64_t *vw;
} orc_owned_graph;

static void owned_free(orc_owned_graph *c) {
  free(c->row_ptr);
  free(c->col);
  free(c->ew);
  free(c->vw);
  memset(c, 0, sizeof(*c));
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* The distinct coarse neighbours y != x of cluster x with their summed
 * weights (sorted by y) into touched[0..nt) / acc[touched[t]]; acc must be
 * zero on entry and is left holding the sums (the caller clears them). */
static int64_t coarse_row(const orc_graph *g, const int32_t *C, const int64_t *mem_ptr,
                          const int32_t *members, int64_t x, int64_t *acc, int32_t *touched,
                          int64_t *vw_x) {
  int64_t nt = 0, wx = 0;
  for (int64_t k = mem_ptr[x]; k < mem_ptr[x + 1]; k++) {
    const int64_t v = members[k];
    wx += g->vw[v];
    for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; e++) {
      const int32_t y = C[g->col[e]];
      if (y == x) continue;
      if (acc[y] == 0) touched[nt++] = y;
      acc[y] += g->ew[e];
    }
  }
  qsort(touched, (size_t)nt, 4, cmp_i32);
  *vw_x = wx;
  return nt;
}

static int contract(const orc_graph *g, const int32_t *C, int64_t n_c, orc_owned_graph *out) {
  memset(out, 0, sizeof(*out));
  const int64_t n = g->n;
  const size_t mc = (size_t)(n_c > 0 ? n_c : 1), nthr = (size_t)orc_threads();
  int64_t *mem_ptr = calloc(mc + 1, 8); /* members of each cluster (counting sort) */
  int32_t *members = malloc((size_t)(n > 0 ? n : 1) * 4);
  int64_t *acc = calloc(mc * nthr, 8);    /* one n_c-slice per thread */
  int32_t *touched = malloc(mc * nthr * 4);
  out->row_ptr = calloc(mc + 1, 8);
  out->vw = calloc(mc, 8);
  int rc = ORC_OK;
  if (!mem_ptr || !members || !acc || !touched || !out->row_ptr || !out->vw) {
    rc = ORC_ERR_OOM;
    goto done;
  }
  for (int64_t v = 0; v < n; v++) mem_ptr[C[v] + 1]++;
  for (int64_t x = 0; x < n_c; x++) mem_ptr[x + 1] += mem_ptr[x];
  {
    int64_t *fill = malloc(mc * 8);
    if (!fill) {
      rc = ORC_ERR_OOM;
      goto done;
    }
    memcpy(fill, mem_ptr, mc * 8);
    for (int64_t v = 0; v < n; v++) members[fill[C[v]]++] = (int32_t)v;
    free(fill);
  }
  /* pass 1: row lengths and coarse vertex weights */
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t x = 0; x < n_c; x++) {
    int64_t *a = acc + (int64_t)orc_thread() * (int64_t)mc;
    int32_t *t = touched + (int64_t)orc_thread() * (int64_t)mc;
    const int64_t nt = coarse_row(g, C, mem_ptr, members, x, a, t, &out->vw[x]);
    for (int64_t k = 0; k < nt; k++) a[t[k]] = 0;
    out->row_ptr[x + 1] = nt;
  }
  for (int64_t x = 0; x < n_c; x++) out->row_ptr[x + 1] += out->row_ptr[x];
  const int64_t len = out->row_ptr[n_c > 0 ? n_c : 0];
  out->col = malloc((size_t)(len > 0 ? len : 1) * 4);
  out->ew = malloc((size_t)(len > 0 ? len : 1) * 4);
  if (!out->col || !out->ew) {
    rc = ORC_ERR_OOM;
    goto done;
  }
  /* pass 2: the rows, sorted by column */
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t x = 0; x < n_c; x++) {
    int64_t *a = acc + (int64_t)orc_thread() * (int64_t)mc;
    int32_t *t = touched + (int64_t)orc_thread() * (int64_t)mc;
    int64_t wx;
    const int64_t nt = coarse_row(g, C, mem_ptr, members, x, a, t, &wx);
    const int64_t o = out->row_ptr[x];
    for (int64_t k = 0; k < nt; k++) {
      out->col[o + k] = t[k];
      out->ew[o + k] = (int32_t)a[t[k]];
      a[t[k]] = 0;
    }
  }
  out->n = n_c;
  out->nnz = len;
done:
  free(mem_ptr);
  free(members);
  free(acc);
  free(touched);
  if (rc) owned_free(out);
  return rc;
}

/* Public contraction: caller frees with orc_free_graph. */
int orc_contract(const orc_graph *g, const int32_t *C, int64_t n_c, int64_t *out_n, int64_t *out_nnz,
                 int64_t **row_ptr, int32_t **col, int32_t **ew, int64_t **vw) {
  if (!g || !C || n_c < 0) return ORC_ERR_ARG;
  for (int64_t v = 0; v < g->n; v++)
    if (C[v] < 0 || C[v] >= n_c) return ORC_ERR_ARG;
  orc_owned_graph c;
  int rc = contract(g, C, n_c, &c);
  if (rc) return rc;
  *out_n = c.n;
  *out_nnz = c.nnz;
  *row_ptr = c.row_ptr;
  *col = c.col;
  *ew = c.ew;
  *vw = c.vw;
  return ORC_OK;
}

void orc_free(void *p) { free(p); }

/* Relabel C to dense ids 0..k-1, in ascending order of the old id. */
static int64_t compact_labels(int32_t *C, int64_t n) {
  int32_t *newid = malloc((size_t)(n > 0 ? n : 1) * 4);
  if (!newid) return -1;
  for (int64_t x = 0; x < n; x++) newid[x] = -1;
  for (int64_t v = 0; v < n; v++) newid[C[v]] = 0;
  int64_t k = 0;
  for (int64_t x = 0; x < n; x++)
    if (newid[x] == 0) newid[x] = (int32_t)k++;
  for (int64_t v = 0; v < n; v++) C[v] = newid[C[v]];
  free(newid);
  return k;
}

/* ---------------------------------------------------------- Louvain+ --- */

/* Algorithm 1: coarsen (singleton start, LocalMovePasses, stop when every
 * cluster is a singleton, otherwise contract) then uncoarsen (project, and
 * for Louvain+ run LocalMovePasses again).  labels_out gets dense ids.
 * With a constraint clustering B0 (>= 0 per vertex; NULL = none) the
 * coarsening-phase LocalMovePasses are constrained by it (Section V-B):
 * coarse vertex x carries the B common to its members (ORC_MIXED if they
 * disagree), and the uncoarsening phase is unconstrained. */
static int louvain_plus(const orc_graph *g0, const orc_params *p, const int32_t *B0,
                        int32_t *labels_out, orc_result *res, orc_callback cb, void *ctx,
                        int32_t passes_before) {
  int rc = check_params(g0, p);
  if (rc) return rc;
  if (!labels_out || !res) return ORC_ERR_ARG;
  if (B0)
    for (int64_t v = 0; v < g0->n; v++)
      if (B0[v] < 0) return ORC_ERR_ARG;
  memset(res, 0, sizeof(*res));
  tracer tr = {cb, ctx, passes_before};

  int cap = 64, L = 0;
  orc_owned_graph *coarse = calloc((size_t)cap, sizeof(orc_owned_graph)); /* G_1.. */
  int32_t **Cl = calloc((size_t)cap, sizeof(int32_t *)); /* dense C_l of each coarsened level */
  int32_t **Bl = calloc((size_t)cap, sizeof(int32_t *)); /* constraint of each coarse level */
  orc_graph *G = calloc((size_t)cap, sizeof(orc_graph));
  int32_t *cur = NULL;
  if (!coarse || !Cl || !Bl || !G) {
    rc = ORC_ERR_OOM;
    goto out;
  }
  G[0] = *g0;
  for (;;) {
    const int64_t n = G[L].n;
    int32_t *C = malloc((size_t)(n > 0 ? n : 1) * 4);
    if (!C) {
      rc = ORC_ERR_OOM;
      goto out;
    }
    for (int64_t v = 0; v < n; v++) C[v] = (int32_t)v; /* SingletonClustering */
    const int32_t *B = L == 0 ? B0 : (B0 ? Bl[L] : NULL);
    if ((rc = local_move_passes(&G[L], p, B, C, L, ORC_PHASE_COARSEN, &tr, NULL))) {
      free(C);
      goto out;
    }
    const int64_t k = compact_labels(C, n);
    if (k < 0) {
      free(C);
      rc = ORC_ERR_OOM;
      goto out;
    }
    if (k == n) { /* |C_l| = |V_l| */
      /* the best-of clustering of a singleton start with no improvement is
       * the singleton clustering itself; compaction leaves it the identity */
      cur = C;
      break;
    }
    if (L + 1 >= cap) {
      free(C);
      rc = ORC_ERR_ARG; /* more than 63 levels: not reachable for n < 2^31 */
      goto out;
    }
    Cl[L] = C;
    if ((rc = contract(&G[L], C, k, &coarse[L + 1]))) goto out;
    if (B0) { /* B of coarse vertex x: the value its members share */
      int32_t *Bn = malloc((size_t)k * 4);
      uint8_t *seen = calloc((size_t)k, 1);
      if (!Bn || !seen) {
        free(Bn);
        free(seen);
        rc = ORC_ERR_OOM;
        goto out;
      }
      for (int64_t v = 0; v < n; v++) {
        const int32_t x = C[v];
        if (!seen[x]) {
          seen[x] = 1;
          Bn[x] = B[v];
        } else if (Bn[x] != B[v]) {
          Bn[x] = ORC_MIXED;
        }
      }
      free(seen);
      Bl[L + 1] = Bn;
    }
    G[L + 1].n = coarse[L + 1].n;
    G[L + 1].nnz = coarse[L + 1].nnz;
    G[L + 1].row_ptr = coarse[L + 1].row_ptr;
    G[L + 1].col = coarse[L + 1].col;
    G[L + 1].ew = coarse[L + 1].ew;
    G[L + 1].vw = coarse[L + 1].vw;
    if (cb) {
      orc_event ev;
      memset(&ev, 0, sizeof(ev));
      ev.kind = ORC_EV_CONTRACT;
      ev.level = L;
      ev.n = n;
      ev.C = C;
      ev.cn = G[L + 1].n;
      ev.cnnz = G[L + 1].nnz;
      ev.c_row_ptr = G[L + 1].row_ptr;
      ev.c_col = G[L + 1].col;
      ev.c_ew = G[L + 1].ew;
      ev.c_vw = G[L + 1].vw;
      cb(ctx, &ev);
    }
    L++;
  }
  res->levels = L + 1;
  /* uncoarsening: l = L-1 .. 0 */
  for (int l = L - 1; l >= 0; l--) {
    const int64_t n = G[l].n;
    int32_t *C = malloc((size_t)(n > 0 ? n : 1) * 4);
    if (!C) {
      rc = ORC_ERR_OOM;
      goto out;
    }
    for (int64_t v = 0; v < n; v++) C[v] = cur[Cl[l][v]]; /* ProjectCluster */
    free(cur);
    cur = C;
    if (p->uncoarsen)
      if ((rc = local_move_passes(&G[l], p, NULL, C, l, ORC_PHASE_UNCOARSEN, &tr, NULL))) goto out;
  }
  {
    const int64_t n = g0->n;
    const int64_t k = compact_labels(cur, n);
    if (k < 0) {
      rc = ORC_ERR_OOM;
      goto out;
    }
    memcpy(labels_out, cur, (size_t)n * 4);
    res->n_clusters = k;
    int64_t *W = malloc((size_t)(n > 0 ? n : 1) * 8);
    if (!W) {
      rc = ORC_ERR_OOM;
      goto out;
    }
    const i128 phi = objective(g0, p->lam_num, p->lam_den, cur, W);
    free(W);
    split128(phi, &res->phi_hi, &res->phi_lo);
    i128 sw2 = 0, T = 0;
    for (int64_t v = 0; v < n; v++) sw2 += (i128)g0->vw[v] * g0->vw[v];
    for (int64_t e = 0; e < g0->nnz; e++) T += g0->ew[e];
    res->objective = (double)(int64_t)phi / (double)p->lam_den;
    res->modularity = T > 0 ? (double)(int64_t)(phi - (i128)p->lam_num * sw2) /
                                  ((double)p->lam_den * (double)(int64_t)T)
                            : 0.0;
    res->passes_total = tr.passes_total;
  }
out:
  free(cur);
  if (Cl)
    for (int l = 0; l < cap; l++) free(Cl[l]);
  if (Bl)
    for (int l = 0; l < cap; l++) free(Bl[l]);
  free(Bl);
  if (coarse)
    for (int l = 0; l < cap; l++) owned_free(&coarse[l]);
  free(Cl);
  free(coarse);
  free(G);
  return rc;
}

int orc_louvain_plus(const orc_graph *g0, const orc_params *p, int32_t *labels_out, orc_result *res,
                     orc_callback cb, void *ctx) {
  return louvain_plus(g0, p, NULL, labels_out, res, cb, ctx, 0);
}

/* Louvain+ whose coarsening is constrained by the clustering B (Section
 * V-B). */
int orc_louvain_plus_constrained(const orc_graph *g0, const orc_params *p, const int32_t *B,
                                 int32_t *labels_out, orc_result *res, orc_callback cb,
                                 void *ctx) {
  if (!B && g0 && g0->n > 0) return ORC_ERR_ARG;
  return louvain_plus(g0, p, B, labels_out, res, cb, ctx, 0);
}

/* Iterated Louvain+ (Section V-B): the first iteration is unconstrained;
 * every further one is constrained by the previous iteration's output.
 * `iterations` >= 1 in total; res describes the last one, with
 * passes_total summed over all. */
int orc_louvain_plus_iterated(const orc_graph *g0, const orc_params *p, int32_t iterations,
                              int32_t *labels_out, orc_result *res, orc_callback cb, void *ctx) {
  if (!g0 || iterations < 1 || !labels_out || !res) return ORC_ERR_ARG;
  int32_t *B = malloc((size_t)(g0->n > 0 ? g0->n : 1) * 4);
  if (!B) return ORC_ERR_OOM;
  int rc = louvain_plus(g0, p, NULL, labels_out, res, cb, ctx, 0);
  for (int32_t it = 1; rc == ORC_OK && it < iterations; it++) {
    memcpy(B, labels_out, (size_t)g0->n * 4);
    rc = louvain_plus(g0, p, B, labels_out, res, cb, ctx, res->passes_total);
  }
  free(B);
  return rc;
}

/* ============================================================ pLeiden ===
 * Section V (Algorithms 5 and 6): pLeiden and pLeiden+.  The random choices
 * of pLeidenR are drawn from a counter-based generator both sides implement
 * from its published definition, so runs are reproducible. */

/* SplitMix64's output function (Steele, Lea and Flood, 2014). */
static uint64_t sm64_mix(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

/* Value number c of the stream (seed, level, stream): SplitMix64's output
 * for state key + (c + 1) * golden gamma, key derived from the stream. */
uint64_t orc_rand(uint32_t seed, int32_t level, int32_t stream, int64_t c) {
  const uint64_t key =
      sm64_mix(((uint64_t)seed << 32) ^ ((uint64_t)(uint32_t)level << 8) ^ (uint64_t)(uint32_t)stream);
  return sm64_mix(key + (uint64_t)(c + 1) * 0x9E3779B97F4A7C15ull);
}

/* LocalMoveAlt (Section V-A): every vertex that is not node-optimal (its
 * ideal destination D[v], chosen by Algorithm 2's rules, has a strictly
 * larger gain than staying) is listed in ascending vertex order.  The moves
 * are applied one after another; the k-th move's exact objective change is
 * taken after all earlier moves of the list (adjacent or not).  The prefix
 * with the largest total change (the shortest among equals) is committed.
 * A move to the empty cluster takes the smallest id unused at that moment;
 * a vertex already alone keeps its id.  Returns the number committed. */
static int64_t local_move_alt(const orc_graph *g, const orc_params *p, int32_t *C, work *w) {
  const int64_t n = g->n, mu = p->lam_num, Lam = p->lam_den;
  cluster_weights(g, C, w->W);
  int64_t m = 0;
  for (int64_t v = 0; v < n; v++) {
    int64_t nt = 0;
    for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; e++) {
      const int32_t X = C[g->col[e]];
      if (w->acc[X] == 0) w->touched[nt++] = X;
      w->acc[X] += g->ew[e];
    }
    const int32_t Cv = C[v];
    const int64_t wv = g->vw[v];
    const i128 gC = (i128)Lam * w->acc[Cv] - (i128)mu * wv * (w->W[Cv] - wv);
    int32_t best = ORC_NONE;
    i128 gbest = 0;
    for (int64_t t = 0; t < nt; t++) {
      const int32_t X = w->touched[t];
      if (X == Cv) continue;
      const i128 gX = (i128)Lam * w->acc[X] - (i128)mu * wv * w->W[X];
      if (best == ORC_NONE || gX > gbest || (gX == gbest && X < best)) {
        best = X;
        gbest = gX;
      }
    }
    for (int64_t t = 0; t < nt; t++) w->acc[w->touched[t]] = 0;
    if (gC < 0 && (best == ORC_NONE || gbest < 0)) {
      best = ORC_EMPTY;
      gbest = 0;
    }
    w->D[v] = best;
    if (best != ORC_NONE && gbest > gC) w->C_next[m++] = (int32_t)v; /* the list, ascending */
  }
  if (m == 0) return 0;
  /* sequential application: W, cluster sizes and labels follow the moves */
  int64_t *size = w->q; /* reused scratch */
  for (int64_t x = 0; x < n; x++) size[x] = 0;
  for (int64_t v = 0; v < n; v++) size[C[v]]++;
  memcpy(w->C_before, C, (size_t)n * sizeof(int32_t));
  int32_t *to = w->mark; /* label taken by the k-th move */
  i128 cum = 0, best_cum = 0;
  int64_t best_k = 0;
  for (int64_t k = 0; k < m; k++) {
    const int32_t v = w->C_next[k], Dv = w->D[v], Cv = C[v];
    const int64_t wv = g->vw[v];
    int64_t Sc = 0, Sd = 0;
    for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; e++) {
      const int32_t X = C[g->col[e]];
      if (X == Cv) Sc += g->ew[e];
      if (Dv >= 0 && X == Dv) Sd += g->ew[e];
    }
    const i128 gC = (i128)Lam * Sc - (i128)mu * wv * (w->W[Cv] - wv);
    const i128 gD = Dv >= 0 ? (i128)Lam * Sd - (i128)mu * wv * w->W[Dv] : 0;
    cum += 2 * (gD - gC);
    if (cum > best_cum) {
      best_cum = cum;
      best_k = k + 1;
    }
    int32_t t = Dv;
    if (Dv == ORC_EMPTY) {
      if (size[Cv] == 1) {
        t = Cv;
      } else {
        int32_t x = 0;
        while (size[x] != 0) x++; /* an unused id exists: a cluster has >= 2 members */
        t = x;
      }
    }
    to[k] = t;
    w->W[Cv] -= wv;
    w->W[t] += wv;
    size[Cv]--;
    size[t]++;
    C[v] = t;
  }
  memcpy(C, w->C_before, (size_t)n * sizeof(int32_t));
  for (int64_t k = 0; k < best_k; k++) C[w->C_next[k]] = to[k];
  return best_k;
}

/* Effective ordering key of pLeidenR: (f, id), compared lexicographically. */
static int key_less(uint64_t fa, int64_t a, uint64_t fb, int64_t b) {
  return fa < fb || (fa == fb && a < b);
}

typedef struct {
  int64_t root;
  uint64_t f;
  int64_t v;
} tree_item;

static int cmp_tree_item(const void *pa, const void *pb) {
  const tree_item *a = (const tree_item *)pa, *b = (const tree_item *)pb;
  if (a->root != b->root) return a->root < b->root ? -1 : 1;
  if (a->f != b->f) return a->f < b->f ? -1 : 1;
  return a->v < b->v ? -1 : (a->v > b->v);
}

/* pLeidenR (Algorithm 6) with constraint clustering B: refined labels R
 * (each vertex gets the id of its cluster's tree root, or its own id).
 *   U: vertices with w'(u, B[u] minus u) >= 0 (Lambda-scaled g(u, B[u]) >= 0).
 *   H[v]: for v in U, a uniformly chosen candidate among v itself and the
 *     neighbours u in U with B[u] = B[v] and w'(u,v) = w(u,v) - lambda
 *     w(u) w(v) >= 0: the one with the smallest (value (v << 32 | c) of
 *     stream 0, c), so the choice does not depend on the order of the row
 *     (coarse rows have none); v itself = no edge.
 *   f(v) in [0, K), K = 2^62: value of stream 1, shifted right by 2.
 *   The edge v -> H[v] is kept iff (f(H[v]), H[v]) < (f(v), v).  A vertex
 *   with an edge that is neither kept nor any kept edge's target (a
 *   singleton tree that did not choose itself) takes f = 2K - f and its
 *   edge is tested again against its target's (possibly changed) key.
 *   Trees are followed to their roots; each tree is visited in increasing
 *   (f, id) (parents come first), and vertex t_k joins the cluster of
 *   t_1..t_(k-1) while w'(t_k, cluster) >= 0 and w'(cluster, B minus
 *   cluster) >= 0 (Leiden's well-connectedness); from the first failure on
 *   the tree's vertices stay singletons. */
static int pleiden_refine(const orc_graph *g, const orc_params *p, const int32_t *B, int32_t level,
                          int32_t *R) {
  const int64_t n = g->n, mu = p->lam_num, Lam = p->lam_den;
  const size_t m = (size_t)(n > 0 ? n : 1);
  int64_t *WB = calloc(m, 8), *SB = calloc(m, 8), *H = malloc(m * 8), *root = malloc(m * 8);
  int64_t *pos = malloc(m * 8);
  uint64_t *f = malloc(m * 8);
  uint8_t *inU = calloc(m, 1), *kept = calloc(m, 1), *child = calloc(m, 1);
  tree_item *items = malloc(m * sizeof(tree_item));
  int rc = ORC_OK;
  if (!WB || !SB || !H || !root || !pos || !f || !inU || !kept || !child || !items) {
    rc = ORC_ERR_OOM;
    goto out;
  }
  const uint64_t K = (uint64_t)1 << 62;
  for (int64_t v = 0; v < n; v++) WB[B[v]] += g->vw[v];
  for (int64_t v = 0; v < n; v++) {
    for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; e++)
      if (B[g->col[e]] == B[v]) SB[v] += g->ew[e];
    inU[v] = (i128)Lam * SB[v] - (i128)mu * g->vw[v] * (WB[B[v]] - g->vw[v]) >= 0;
    f[v] = orc_rand(p->seed, level, 1, v) >> 2;
  }
  for (int64_t v = 0; v < n; v++) {
    H[v] = v;
    if (!inU[v]) continue;
    /* ChooseRandom: the candidate c (v itself or a qualifying neighbour)
     * with the smallest (rand(v, c), c); uniform over the candidates and
     * independent of the order of the row. */
    uint64_t best = orc_rand(p->seed, level, 0, (v << 32) | v);
    for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; e++) {
      const int64_t u = g->col[e];
      if (inU[u] && B[u] == B[v] &&
          (i128)Lam * g->ew[e] - (i128)mu * g->vw[u] * g->vw[v] >= 0) {
        const uint64_t r = orc_rand(p->seed, level, 0, (v << 32) | u);
        if (r < best || (r == best && u < H[v])) {
          best = r;
          H[v] = u;
        }
      }
    }
  }
  for (int64_t v = 0; v < n; v++) {
    kept[v] = H[v] != v && key_less(f[H[v]], H[v], f[v], v);
    if (kept[v]) child[H[v]] = 1;
  }
  for (int64_t v = 0; v < n; v++) /* singleton trees that chose an edge */
    if (H[v] != v && !kept[v] && !child[v]) f[v] = 2 * K - f[v];
  for (int64_t v = 0; v < n; v++)
    if (H[v] != v && !kept[v] && !child[v]) kept[v] = key_less(f[H[v]], H[v], f[v], v);
  for (int64_t v = 0; v < n; v++) {
    int64_t r = v, steps = 0;
    while (kept[r]) {
      r = H[r];
      if (++steps > n) { /* impossible: keys strictly decrease along kept edges */
        rc = ORC_ERR_ARG;
        goto out;
      }
    }
    root[v] = r;
  }
  for (int64_t v = 0; v < n; v++) items[v] = (tree_item){root[v], f[v], v};
  qsort(items, (size_t)n, sizeof(tree_item), cmp_tree_item);
  for (int64_t i = 0; i < n; i++) pos[items[i].v] = i;
  for (int64_t i = 0; i < n;) {
    int64_t j = i;
    while (j < n && items[j].root == items[i].root) j++;
    const int64_t r = items[i].root;
    const int64_t t1 = items[i].v;
    R[t1] = (int32_t)t1;
    int64_t Wc = g->vw[t1], Ec = SB[t1];
    int ok = 1;
    for (int64_t k = i + 1; k < j; k++) {
      const int64_t v = items[k].v;
      if (ok) {
        int64_t Sv = 0; /* edges to the earlier vertices of the tree */
        for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; e++) {
          const int64_t u = g->col[e];
          if (root[u] == r && pos[u] < k) Sv += g->ew[e];
        }
        const int c1 = (i128)Lam * Sv - (i128)mu * g->vw[v] * Wc >= 0;
        const int c2 = (i128)Lam * Ec - (i128)mu * Wc * (WB[B[v]] - Wc) >= 0;
        if (c1 && c2) {
          R[v] = (int32_t)t1;
          Ec += SB[v] - 2 * Sv;
          Wc += g->vw[v];
          continue;
        }
        ok = 0;
      }
      R[v] = (int32_t)v;
    }
    i = j;
  }
out:
  free(WB);
  free(SB);
  free(H);
  free(root);
  free(pos);
  free(f);
  free(inU);
  free(kept);
  free(child);
  free(items);
  return rc;
}

/* pLeiden (Algorithm 5); with p->uncoarsen, pLeiden+ (LocalMovePasses
 * after each projection).  C_in: initial clustering (labels in [0, n)),
 * NULL for singletons.  Per level: LocalMovePasses from C_l; LocalMoveAlt
 * when they left Phi unchanged; stop when every cluster is a singleton;
 * otherwise refine (pLeidenR with B = C_l, the level as stream), contract
 * on the refinement, and Downsample: coarse vertex x starts in the cluster
 * of C_l its members share.  A refinement that merges nothing also ends
 * the coarsening (contracting it would reproduce G_l).  labels_out gets
 * dense ids; res as for orc_louvain_plus. */
int orc_pleiden(const orc_graph *g0, const orc_params *p, const int32_t *C_in, int32_t *labels_out,
                orc_result *res, orc_callback cb, void *ctx) {
  int rc = check_params(g0, p);
  if (rc) return rc;
  if (!labels_out || !res) return ORC_ERR_ARG;
  if (C_in)
    for (int64_t v = 0; v < g0->n; v++)
      if (C_in[v] < 0 || C_in[v] >= g0->n) return ORC_ERR_ARG;
  memset(res, 0, sizeof(*res));
  tracer tr = {cb, ctx, 0};
  int cap = 64, L = 0;
  orc_owned_graph *coarse = calloc((size_t)cap, sizeof(orc_owned_graph));
  int32_t **Rl = calloc((size_t)cap, sizeof(int32_t *)); /* dense refinement of each level */
  orc_graph *G = calloc((size_t)cap, sizeof(orc_graph));
  int32_t *C = NULL;
  work w;
  memset(&w, 0, sizeof(w));
  if (!coarse || !Rl || !G) {
    rc = ORC_ERR_OOM;
    goto out;
  }
  G[0] = *g0;
  C = malloc((size_t)(g0->n > 0 ? g0->n : 1) * 4);
  if (!C) {
    rc = ORC_ERR_OOM;
    goto out;
  }
  for (int64_t v = 0; v < g0->n; v++) C[v] = C_in ? C_in[v] : (int32_t)v;
  for (;;) {
    const int64_t n = G[L].n;
    i128 phi_in = 0, phi_out = 0;
    {
      int64_t *Ws = malloc((size_t)(n > 0 ? n : 1) * 8);
      if (!Ws) {
        rc = ORC_ERR_OOM;
        goto out;
      }
      phi_in = objective(&G[L], p->lam_num, p->lam_den, C, Ws);
      free(Ws);
    }
    if ((rc = local_move_passes(&G[L], p, NULL, C, L, ORC_PHASE_COARSEN, &tr, &phi_out))) goto out;
    if (phi_out == phi_in) {
      if (work_alloc(&w, n)) {
        rc = ORC_ERR_OOM;
        goto out;
      }
      local_move_alt(&G[L], p, C, &w);
      work_free(&w);
    }
    const int64_t k = compact_labels(C, n);
    if (k < 0) {
      rc = ORC_ERR_OOM;
      goto out;
    }
    if (k == n) break;
    if (L + 1 >= cap) {
      rc = ORC_ERR_ARG;
      goto out;
    }
    int32_t *R = malloc((size_t)n * 4);
    if (!R) {
      rc = ORC_ERR_OOM;
      goto out;
    }
    if ((rc = pleiden_refine(&G[L], p, C, L, R))) {
      free(R);
      goto out;
    }
    const int64_t kr = compact_labels(R, n);
    if (kr < 0 || kr == n) {
      free(R);
      if (kr < 0) rc = ORC_ERR_OOM;
      if (rc) goto out;
      break;
    }
    Rl[L] = R;
    if ((rc = contract(&G[L], R, kr, &coarse[L + 1]))) goto out;
    G[L + 1].n = coarse[L + 1].n;
    G[L + 1].nnz = coarse[L + 1].nnz;
    G[L + 1].row_ptr = coarse[L + 1].row_ptr;
    G[L + 1].col = coarse[L + 1].col;
    G[L + 1].ew = coarse[L + 1].ew;
    G[L + 1].vw = coarse[L + 1].vw;
    if (cb) {
      orc_event ev;
      memset(&ev, 0, sizeof(ev));
      ev.kind = ORC_EV_CONTRACT;
      ev.level = L;
      ev.n = n;
      ev.C = R;
      ev.cn = G[L + 1].n;
      ev.cnnz = G[L + 1].nnz;
      ev.c_row_ptr = G[L + 1].row_ptr;
      ev.c_col = G[L + 1].col;
      ev.c_ew = G[L + 1].ew;
      ev.c_vw = G[L + 1].vw;
      cb(ctx, &ev);
    }
    /* Downsample: coarse vertex x starts in the C_l cluster of its members */
    int32_t *Cn = malloc((size_t)kr * 4);
    if (!Cn) {
      rc = ORC_ERR_OOM;
      goto out;
    }
    for (int64_t v = 0; v < n; v++) Cn[R[v]] = C[v];
    if (compact_labels(Cn, kr) < 0) {
      free(Cn);
      rc = ORC_ERR_OOM;
      goto out;
    }
    free(C);
    C = Cn;
    L++;
  }
  res->levels = L + 1;
  for (int l = L - 1; l >= 0; l--) { /* ProjectCluster, and for pLeiden+ LocalMovePasses */
    const int64_t n = G[l].n;
    int32_t *Cp = malloc((size_t)(n > 0 ? n : 1) * 4);
    if (!Cp) {
      rc = ORC_ERR_OOM;
      goto out;
    }
    for (int64_t v = 0; v < n; v++) Cp[v] = C[Rl[l][v]];
    free(C);
    C = Cp;
    if (p->uncoarsen)
      if ((rc = local_move_passes(&G[l], p, NULL, C, l, ORC_PHASE_UNCOARSEN, &tr, NULL))) goto out;
  }
  {
    const int64_t n = g0->n;
    const int64_t k = compact_labels(C, n);
    int64_t *W = malloc((size_t)(n > 0 ? n : 1) * 8);
    if (k < 0 || !W) {
      free(W);
      rc = ORC_ERR_OOM;
      goto out;
    }
    memcpy(labels_out, C, (size_t)n * 4);
    res->n_clusters = k;
    const i128 phi = objective(g0, p->lam_num, p->lam_den, C, W);
    free(W);
    split128(phi, &res->phi_hi, &res->phi_lo);
    i128 sw2 = 0, T = 0;
    for (int64_t v = 0; v < n; v++) sw2 += (i128)g0->vw[v] * g0->vw[v];
    for (int64_t e = 0; e < g0->nnz; e++) T += g0->ew[e];
    res->objective = (double)(int64_t)phi / (double)p->lam_den;
    res->modularity = T > 0 ? (double)(int64_t)(phi - (i128)p->lam_num * sw2) /
                                  ((double)p->lam_den * (double)(int64_t)T)
                            : 0.0;
    res->passes_total = tr.passes_total;
  }
out:
  work_free(&w);
  free(C);
  if (Rl)
    for (int l = 0; l < cap; l++) free(Rl[l]);
  if (coarse)
    for (int l = 0; l < cap; l++) owned_free(&coarse[l]);
  free(Rl);
  free(coarse);
  free(G);
  return rc;
}

/* Test hooks: one LocalMoveAlt call and one pLeidenR call on level `level`. */
int orc_local_move_alt(const orc_graph *g, const orc_params *p, int32_t *C, int64_t *committed) {
  int rc = check_params(g, p);
  if (rc) return rc;
  for (int64_t v = 0; v < g->n; v++)
    if (C[v] < 0 || C[v] >= g->n) return ORC_ERR_ARG;
  work w;
  if (work_alloc(&w, g->n)) return ORC_ERR_OOM;
  const int64_t k = local_move_alt(g, p, C, &w);
  work_free(&w);
  if (committed) *committed = k;
  return ORC_OK;
}

int orc_pleiden_refine(const orc_graph *g, const orc_params *p, const int32_t *B, int32_t level,
                       int32_t *R) {
  int rc = check_params(g, p);
  if (rc) return rc;
  for (int64_t v = 0; v < g->n; v++)
    if (B[v] < 0 || B[v] >= g->n) return ORC_ERR_ARG;
  return pleiden_refine(g, p, B, level, R);
}
