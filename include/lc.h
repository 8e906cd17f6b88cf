/*
 * lc.h — C ABI of the GB300 (sm_103a) pLouvain / Louvain+ library, liblc.so.
 *
 * The library clusters an undirected graph by optimising the LambdaCC
 * objective (Gilbert & Madduri, "GPU-Accelerated Multilevel Graph Clustering:
 * A Parallel Perspective on Louvain and Leiden", Section II-A, Eq. 1):
 *
 *   lambdaCC(C) = sum over clusters C_i, over ordered pairs u != v in C_i,
 *                 of ( w(u,v) - lambda * w(u) * w(v) )
 *
 * with positive integer vertex weights w(v), positive integer edge weights
 * w(u,v) and a rational lambda = lambda_num / lambda_den in [0, 1].
 * Modularity is the special case w(v) = weighted degree and
 * lambda = gamma / (sum of all stored edge weights); the Constant Potts
 * Model is w(v) = 1 (Section II-A).
 *
 * The method is Louvain+ (Algorithm 1): coarsening levels of synchronous
 * local-move passes (Algorithm 2) filtered by the afterburner (Algorithm 3),
 * gather-free graph contraction (Algorithm 4), then uncoarsening levels that
 * project and re-run the local-move passes.  Also: Louvain+ constrained by a
 * clustering and its iterated form (Section V-B), and pLeiden / pLeiden+
 * (Section V).  All arithmetic is exact integer; results are deterministic
 * and independent of thread scheduling.
 *
 * Conventions shared by every entry point:
 *  - Graphs are CSR: row_ptr int64[n+1] (row_ptr[0] = 0, row_ptr[n] = nnz,
 *    non-decreasing), col int32[nnz] in [0, n), edge weights int32[nnz] > 0.
 *    Both directions of every undirected edge are stored with equal weight;
 *    rows are strictly increasing (sorted, no duplicates); no self-loops.
 *  - Vertex weights int64[n] >= 0 (Section II asks for positive weights; zero
 *    is also accepted, the modularity weight of an isolated vertex).
 *    0 <= lambda_num <= lambda_den, lambda_den > 0.
 *  - Unless an entry point says "host", every pointer argument that refers
 *    to graph or label data is DEVICE memory on the current CUDA device,
 *    owned by the caller, read-only unless it is an output, and not retained
 *    after the call returns.  Work is issued on opts->stream (NULL = the
 *    legacy default stream); every call returns after its results are
 *    complete on that stream (calls read per-level sizes back to the host).
 *  - Scratch device memory comes from opts->alloc / opts->dealloc when the
 *    caller sets them (the Python binding passes PyTorch's caching
 *    allocator), else from a stream-ordered memory pool private to the
 *    library (cudaMemPoolCreate; the device's default pool is never
 *    touched).  Either way every scratch buffer is returned before the call
 *    returns: to the caller's allocator, or to the private pool, which keeps
 *    the freed blocks cached for later calls until lc_release_memory().
 *  - Return value: LC_OK or an LC_ERR_* code; on error no output is
 *    guaranteed to have been written (labels_out may hold partial data) and
 *    *res is zeroed except for res->error_detail.  lc_strerror() names it.
 *  - Exactness guards (checked before any work, LC_ERR_OVERFLOW):
 *    T = sum of edge weights < 2^31 and, with V = sum of vertex weights,
 *    B = lambda_den*T + lambda_num*V^2 < 2^60, and
 *    (eps_den/eps_num) * 2 * (T + lambda_num*V^2/lambda_den) < 2^60.
 */
#ifndef LC_H
#define LC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LC_API __attribute__((visibility("default")))
#else
#define LC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
  LC_OK = 0,
  LC_ERR_ARG = 1,        /* bad argument, size or option */
  LC_ERR_ASYMMETRIC = 2, /* some (u,v,w) has no matching (v,u,w) */
  LC_ERR_SELF_LOOP = 3,  /* some row v lists v */
  LC_ERR_DUPLICATE = 4,  /* a row is not strictly increasing */
  LC_ERR_WEIGHT = 5,     /* an edge weight <= 0 or a vertex weight < 0 */
  LC_ERR_OVERFLOW = 6,   /* exactness guard tripped (see above) */
  LC_ERR_OOM = 7,        /* device allocation failed */
  LC_ERR_CUDA = 8,       /* a CUDA runtime call failed */
  LC_ERR_TIMEOUT = 9,    /* level cap (256) reached */
  LC_ERR_DEVICE = 10,    /* a kernel reported an internal bound violation */
  LC_ERR_NOT_READY = 11  /* server: job still running */
};

/* Graph topology: n vertices, nnz stored (directed) entries. */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int64_t *row_ptr; /* [n+1] */
  const int32_t *col;     /* [nnz] */
} lc_csr;

/* Trace record delivered to lc_opts.event_cb (host copies, valid during the
 * callback only).  Used to compare every pass and level with a reference. */
enum { LC_EV_PASS = 1, LC_EV_LMP = 2, LC_EV_CONTRACT = 3 };
typedef struct {
  int32_t kind;   /* LC_EV_* */
  int32_t level;  /* graph level l (0 = input) */
  int32_t phase;  /* 0 coarsening, 1 uncoarsening */
  int32_t pass;   /* 1-based pass index (PASS only) */
  int64_t n;      /* vertices of G_l */
  const int32_t *labels; /* PASS: C after the pass; LMP: C_out; CONTRACT: dense C */
  const int32_t *dest;   /* PASS: D[v] for candidates, -1 non-candidate, -2 empty cluster */
  const uint8_t *moved;  /* PASS: 1 if v passed the afterburner */
  int64_t phi;           /* PASS: Phi(C after pass); LMP: Phi(C_out) (Phi = lambda_den*lambdaCC) */
  int64_t count_L, count_M;
  int64_t cn, cnnz;      /* CONTRACT: coarse graph G_{l+1} (rows unsorted) */
  const int64_t *c_row_ptr;
  const int32_t *c_col;
  const int32_t *c_ew;
  const int64_t *c_vw;
} lc_event;
typedef void (*lc_event_fn)(void *ctx, const lc_event *ev);

/* Device memory provider of lc_opts (optional; both or neither).
 * alloc returns `bytes` of device memory on the current device that may be
 * used in the order of `stream` (the cudaStream_t of the call), or NULL if
 * it has none, which fails the call with LC_ERR_OOM after everything it
 * took is given back.  dealloc returns a block in the order of the same
 * stream; the library calls it once per block, before the call that took
 * the block returns.  ctx is lc_opts.alloc_ctx.  Server slots call these
 * from their own threads, so a provider given to lc_server_create must be
 * thread-safe. */
typedef void *(*lc_alloc_fn)(void *ctx, size_t bytes, void *stream);
typedef void (*lc_free_fn)(void *ctx, void *ptr, size_t bytes, void *stream);

/* Options.  Initialise with lc_default_opts(). */
typedef struct {
  int32_t pass_limit;       /* passes per LocalMovePasses call (Algorithm 2); default 6, max 16 */
  int32_t phi_num[16];      /* temperature phi_i = phi_num[i]/phi_den[i] of pass i+1 */
  int32_t phi_den[16];      /* default 3/4 for passes 1-4, 1/4 for passes 5-6 (Section VI-C) */
  int32_t eps_num, eps_den; /* epsilon of the afterburner ordering (Section IV-A-1); default 1/10 */
  uint32_t seed;            /* salt of the ordering hash; default 0 */
  int32_t uncoarsen;        /* 1 = Louvain+ (default), 0 = Louvain (Algorithm 1 line 12 off) */
  int32_t validate;         /* 1 = check the CSR preconditions on the device (default) */
  int32_t profile;          /* 1 = time each kernel class with CUDA events into lc_result */
  void *stream;             /* cudaStream_t */
  lc_event_fn event_cb;     /* optional per-pass / per-level trace (slow: syncs and copies) */
  void *event_ctx;
  int32_t symmetry;         /* symmetry breaking of the passes: 0 = afterburner filter
                               (Algorithm 3, default); 1 = none, every candidate moves;
                               2 = minimum label heuristic in odd passes (a vertex alone in
                               its cluster may not join another one-vertex cluster with a
                               larger label), none in even passes.  1 and 2 are the
                               ablations of Section VI. */
  int32_t tables;           /* how the passes get S(v, .) (Algorithm 2): 0 = every pass
                               aggregates it from the CSR (default); 1 = vertices of
                               degree above 256 keep their tables across the passes of a
                               LocalMovePasses call, and each later pass updates them in
                               place from the last pass's movers (Section IV-A-3).
                               Results are identical; 0 is faster on the graphs measured. */
  int64_t scratch_limit;    /* bytes of device scratch one call may hold at once; 0 = no
                               limit.  A call that needs more returns LC_ERR_OOM (nothing
                               is kept allocated), as when the device itself runs out. */
  lc_alloc_fn alloc;        /* device scratch provider (see lc_alloc_fn); NULL together
                               with dealloc = the library's private pool (default) */
  lc_free_fn dealloc;
  void *alloc_ctx;          /* passed to alloc and dealloc */
  int32_t bin_max_deg[9];   /* degree bins of the per-vertex kernels (the degree buckets of
                               Section IV-C-2, whose thresholds the paper leaves open):
                               bin k takes bin_max_deg[k-1] < deg <= bin_max_deg[k], rows
                               above bin_max_deg[8] are "hubs" cut into hub_chunk-edge
                               chunks.  0 = the default of that bin (8, 16, 32, 128, 256,
                               512, 1024, 2048, 4096, which are also each bin's largest
                               allowed value); equal neighbours leave a bin empty.  Values
                               must be non-decreasing (LC_ERR_ARG otherwise).  Results do
                               not depend on them; lc_autotune picks them by timing.
                               opts.tables = 1 needs the defaults. */
  int32_t hub_chunk;        /* edges per hub chunk; 0 = 2048; 256 .. 65536 */
  int32_t ab_threads[5];    /* threads per candidate in the afterburner's launch groups
                               (bin 0, bin 1, bins 2-4, bins 5-6, bins 7-8): 0 = the
                               default (1, 16, 32, 128, 512); groups 2-4 also take 32, 128
                               or 512, group 2 also 16.  Results do not depend on them. */
  int32_t graphs;           /* 1 = the passes of a LocalMovePasses call that repeat the same
                               launches (all but a first pass from singletons and the last)
                               are captured once per call into a CUDA graph and replayed,
                               which removes most per-kernel launch costs on small graphs.
                               Ignored with profile, event_cb or tables = 1.  Results are
                               identical.  Default 0. */
} lc_opts;

/* Kernel classes timed when opts.profile = 1. */
enum {
  LC_K_FIRST_PASS = 0, /* first-pass argmax straight from the CSR (Section IV-A-3) */
  LC_K_MOVE = 1,       /* neighbour-cluster aggregation + gain argmax + candidate test */
  LC_K_AFTERBURNER = 2,
  LC_K_APPLY = 3,      /* update + new-singleton ids + best-of copy */
  LC_K_OBJECTIVE = 4,
  LC_K_CONTRACT = 5,   /* label compaction + contraction */
  LC_K_OTHER = 6,      /* binning, projection, validation, guards */
  LC_K_ALT = 7,        /* pLeiden: LocalMoveAlt (Section V-A) */
  LC_K_REFINE = 8,     /* pLeiden: pLeidenR refinement (Algorithm 6) */
  LC_K_TABLE = 9,      /* kept tables: in-place update from the movers + argmax and
                          candidate test read from the tables (Section IV-A-3) */
  LC_K_COUNT = 10
};

typedef struct {
  int64_t n_clusters;
  int32_t levels;       /* number of graphs G_0..G_top */
  int32_t passes_total; /* local-move passes run, all levels and phases */
  int64_t phi;          /* exact Phi = lambda_den * lambdaCC(labels) */
  int64_t lambda_den;
  double objective;     /* lambdaCC = phi / lambda_den */
  double modularity;    /* (phi - lambda_num*sum w(v)^2) / (lambda_den * sum w(u,v));
                           the modularity when w(v) is the weighted degree */
  int64_t edges_local_move; /* sum over passes of nnz(G_l) */
  int64_t edges_contract;   /* sum over contractions of nnz(G_l) */
  /* opts.profile = 1: per kernel class, total milliseconds, launches and
   * algorithmic bytes (the minimum bytes the kernels must move) */
  double kernel_ms[LC_K_COUNT];
  int64_t kernel_launches[LC_K_COUNT];
  double kernel_bytes[LC_K_COUNT];
  int64_t error_detail; /* extra context for some errors (e.g. offending vertex) */
  int64_t tables_rebuilt; /* kept tables (opts.tables) that ran out of slots during an
                             in-place update and were rebuilt from the labels */
  int64_t scratch_peak_bytes; /* most device scratch the call held at once (bytes
                                 requested from the provider) */
} lc_result;

/* Fill *o with the defaults of Section VI-C (pass limit 6, phi 3/4 x4 then
 * 1/4 x2, epsilon 1/10, seed 0, Louvain+, validate on, profile off). */
LC_API void lc_default_opts(lc_opts *o);

/* Upper estimate, in bytes, of the device scratch lc_cluster (count = 1) or
 * lc_cluster_batch (count graphs) needs on a graph of n vertices and nnz
 * stored edges: the level-0 scratch exactly, the sizes the driver requests,
 * plus coarse levels whose vertex and edge counts sum to at most those of
 * the input.  A run whose levels shrink more slowly can need more (compare
 * lc_result.scratch_peak_bytes).  -1 for negative sizes or count < 1. */
LC_API int64_t lc_scratch_estimate(int64_t n, int64_t nnz, int32_t count, const lc_opts *opts);

/* LC_OK if *opts is a valid option set for the clustering calls (pass limit
 * and schedule, epsilon, symmetry and table modes, scratch limit, both or
 * neither of alloc / dealloc, graphs, and the launch settings bin_max_deg /
 * hub_chunk / ab_threads with their rules above), else LC_ERR_ARG; null
 * opts: the defaults.  Host arithmetic only: needs no device. */
LC_API int lc_check_opts(const lc_opts *opts);

/* Launch settings chosen by lc_autotune. */
typedef struct {
  int32_t bin_max_deg[9]; /* for lc_opts.bin_max_deg */
  int32_t hub_chunk;      /* for lc_opts.hub_chunk */
  int32_t ab_threads[5];  /* for lc_opts.ab_threads */
  int32_t graphs;         /* for lc_opts.graphs */
  int32_t trials;         /* settings timed */
  double ms_default;      /* median milliseconds of one call with the starting settings */
  double ms_best;         /* ... with the chosen ones */
} lc_tuning;

/* Picks the degree-bin boundaries, hub chunk length, afterburner thread
 * groups and graph replay for a
 * workload by timing them (the paper leaves its bucket thresholds open,
 * Section IV-C-2; no setting changes a result).  Starting from opts (NULL:
 * the defaults), it moves one setting at a time, runs lc_cluster (count = 1)
 * or lc_cluster_batch (count graphs, as that call) `repeats` times after one
 * untimed run, and keeps a change only if the median time falls.  Every
 * candidate's labels are compared with those of the starting settings
 * (LC_ERR_DEVICE if one differs, which would be a library fault).  Arguments
 * as lc_cluster / lc_cluster_batch: graph_ptr, lambda_num and lambda_den are
 * HOST arrays (count + 1, count, count entries); for count = 1 graph_ptr may
 * be NULL.  opts.tables = 1 is rejected (LC_ERR_ARG).  Each trial is a full
 * clustering, so the call takes about 2 * 15 * repeats clusterings. */
LC_API int lc_autotune(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w, int32_t count,
                       const int64_t *graph_ptr, const int64_t *lambda_num, const int64_t *lambda_den,
                       const lc_opts *opts, int32_t repeats, lc_tuning *out);

/* Human-readable name of an LC_* code (static string). */
LC_API const char *lc_strerror(int code);

/* Returns the blocks cached in the library's private memory pool on the
 * current device to the device (cudaMemPoolTrimTo after a device-wide
 * synchronize), e.g. before handing the GPU's memory to another allocator.
 * Later calls grow the pool again.  Memory that opts.alloc provided is never
 * cached by the library.  LC_OK or LC_ERR_CUDA. */
LC_API int lc_release_memory(void);

/* Louvain+ (Algorithm 1) on G = (g, vertex_w, edge_w) with
 * lambda = lambda_num / lambda_den.  labels_out: device int32[n], written
 * with dense cluster ids 0..k-1 numbered in ascending order of the level-0
 * cluster id.  res (host) receives counts, the exact objective and, with
 * opts.profile, kernel timings.  opts may be NULL for the defaults. */
LC_API int lc_cluster(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w, int64_t lambda_num,
               int64_t lambda_den, const lc_opts *opts, int32_t *labels_out, lc_result *res);

/* Louvain+ with a constraint clustering (Section V-B, the note on iterating
 * Louvain+): during coarsening a vertex may only join a cluster whose
 * members all carry its own constraint label, so every coarsening-phase
 * cluster lies inside one class; coarse vertices carry their members'
 * label; the uncoarsening phase is unconstrained.  constraint: device
 * int32[n] (only equality of labels matters), read-only, caller-owned,
 * NULL only when n = 0 (LC_ERR_ARG otherwise).  Everything else as
 * lc_cluster. */
LC_API int lc_cluster_constrained(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                                  int64_t lambda_num, int64_t lambda_den, const int32_t *constraint,
                                  const lc_opts *opts, int32_t *labels_out, lc_result *res);

/* pLeiden (Algorithm 5, Section V) on G; opts.uncoarsen = 1 (the default)
 * gives pLeiden+ (LocalMovePasses after each projection), 0 gives pLeiden.
 * Each level runs LocalMovePasses from its clustering, LocalMoveAlt
 * (Section V-A) when they leave the objective unchanged, then stops if
 * every cluster is a singleton, else refines with pLeidenR (Algorithm 6),
 * contracts on the refinement and starts the coarse level from the
 * clusters (Downsample).  A refinement that merges nothing also ends the
 * coarsening.  pLeidenR's random choices come from SplitMix64's output
 * function on (opts.seed, level, stream, vertex), so runs are reproducible.
 * initial: device int32[n] starting clustering with labels in [0, n)
 * (LC_ERR_ARG otherwise), or NULL for singletons.  labels_out and res as
 * lc_cluster; res.passes_total counts the LocalMovePasses passes. */
LC_API int lc_cluster_leiden(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                             int64_t lambda_num, int64_t lambda_den, const int32_t *initial,
                             const lc_opts *opts, int32_t *labels_out, lc_result *res);

/* Iterated Louvain+ (Section V-B): `iterations` (>= 1) runs in total; the
 * first is lc_cluster, each further one is lc_cluster_constrained with the
 * previous output as the constraint.  labels_out gets the last output; res
 * describes the last run, with passes, edge counts and kernel profile
 * summed over all runs.  Allocates one int32[n] device buffer on
 * opts.stream for the constraint. */
LC_API int lc_cluster_iterated(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                               int64_t lambda_num, int64_t lambda_den, int32_t iterations,
                               const lc_opts *opts, int32_t *labels_out, lc_result *res);

/* Batched Louvain+: `count` independent graphs packed into one CSR g (the
 * disjoint union, global vertex ids): graph k owns the vertex range
 * [graph_ptr[k], graph_ptr[k+1]) (graph_ptr: HOST int64[count+1], 0 first,
 * g->n last) and every edge stays inside its graph (checked with
 * opts.validate, LC_ERR_ARG otherwise).  Each graph has its own
 * lambda_num[k] / lambda_den[k] (HOST int64[count]).  All graphs run through
 * the same kernel launches level by level (a graph that finishes
 * coarsening drops out of the next levels); each graph's result is exactly
 * what lc_cluster returns for it alone.  labels_out: device int32[g->n],
 * labels of graph k numbered 0..k_k-1 within the graph.  res: HOST
 * lc_result[count], one per graph; the kernel timings of opts.profile and
 * the edge counters are call-wide and reported in res[0].  The trace
 * callback is not used by batched calls. */
LC_API int lc_cluster_batch(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                            int32_t count, const int64_t *graph_ptr, const int64_t *lambda_num,
                            const int64_t *lambda_den, const lc_opts *opts, int32_t *labels_out,
                            lc_result *res);

/* Clustering service (the served form).  Requests are host graphs; the
 * server copies them on submit.  `slots` worker threads, each with its own
 * CUDA stream on the device that was current at lc_server_create, admit
 * queued requests in arrival order while their device footprint fits in the
 * unclaimed part of `hbm_budget` (0: half of the free device memory at
 * creation; a request larger than the whole budget runs alone), up to
 * `max_batch` per slot, and cluster each admission as one
 * lc_cluster_batch call.  A request's footprint is its packed input (24
 * bytes per vertex + 8 per stored edge) plus lc_scratch_estimate() for it;
 * an admission's clustering runs with the scratch it reserved as its
 * scratch limit, and if the estimate falls short its requests return to the
 * head of the queue with twice the reservation (LC_ERR_OOM reaches a caller
 * only when the device itself is out of memory).  Slots run concurrently,
 * so requests arriving while others are on the GPU start as soon as a slot
 * and memory free up.  Every job's labels and result equal lc_cluster's for
 * that graph alone.  opts applies to every job (its stream, trace, profile
 * and scratch_limit fields are ignored; its allocator, if set, is called
 * from the slots' threads). */
typedef struct lc_server lc_server;
typedef struct {
  int32_t slots;      /* concurrent admissions (default 4, max 64) */
  int32_t max_batch;  /* jobs per admission (default 64) */
  int64_t hbm_budget; /* bytes; 0 = half of the free device memory */
  lc_opts opts;
} lc_server_config;
LC_API void lc_server_default_config(lc_server_config *c);
LC_API int lc_server_create(const lc_server_config *cfg, lc_server **out);
/* Queue one graph (HOST pointers, copied before return); *job_id names it. */
LC_API int lc_server_submit(lc_server *s, const lc_csr *g_host, const int64_t *vertex_w,
                            const int32_t *edge_w, int64_t lambda_num, int64_t lambda_den,
                            int64_t *job_id);
/* If the job is done: copy its labels (HOST int32[n], may be NULL) and result
 * (may be NULL), report submit-to-done seconds (may be NULL), forget the job
 * and return its status; otherwise LC_ERR_NOT_READY.  A request that breaks
 * a precondition or guard fails alone (its admission is re-run job by job)
 * with that error and res->error_detail; the other jobs are unaffected. */
LC_API int lc_server_poll(lc_server *s, int64_t job_id, int32_t *labels_out, lc_result *res,
                          double *latency_s);
/* Like lc_server_poll but blocks until the job is done. */
LC_API int lc_server_wait(lc_server *s, int64_t job_id, int32_t *labels_out, lc_result *res,
                          double *latency_s);
/* Withdraws a job that is still queued: LC_OK (the id is then unknown),
 * LC_ERR_NOT_READY if it is already running or done (poll or wait for it),
 * LC_ERR_ARG for an unknown id. */
LC_API int lc_server_cancel(lc_server *s, int64_t job_id);
/* Finishes the queued and running jobs, stops the workers, frees the server. */
LC_API int lc_server_destroy(lc_server *s);

/* Same as lc_cluster with HOST buffers (pinned or pageable): copies the graph
 * to the device on opts->stream, clusters it, and copies labels_out (host
 * int32[n]) back before returning. */
LC_API int lc_cluster_host(const lc_csr *g_host, const int64_t *vertex_w, const int32_t *edge_w,
                    int64_t lambda_num, int64_t lambda_den, const lc_opts *opts,
                    int32_t *labels_out, lc_result *res);

/* One LocalMovePasses call (Algorithm 2 with Algorithm 3) from the device
 * clustering labels_inout (int32[n], values in [0, n)), which is replaced by
 * the best clustering seen (C_out).  singleton_start = 1 asserts that the
 * input is the all-singleton clustering labels[v] = v, enabling the
 * first-pass shortcut of Section IV-A-3 (the result is the same). */
LC_API int lc_local_move(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                  int64_t lambda_num, int64_t lambda_den, const lc_opts *opts,
                  int32_t *labels_inout, int32_t singleton_start, lc_result *res);

/* Graph contraction (Algorithm 4; the coarse graph of Section III-A): labels
 * is a device int32[n] clustering with dense ids in [0, n_c).  Writes the
 * coarse graph into caller-allocated device buffers: c_row_ptr int64[n_c+1],
 * c_col int32[cap], c_ew int32[cap], c_vw int64[n_c] with cap >= the number
 * of coarse entries (nnz is always enough); *c_nnz (host) receives the
 * number of entries.  Coarse edge (x,y) has weight w(C_x, C_y) and exists
 * iff it is positive; no self-loops; c_vw[x] = w(C_x); rows are unsorted. */
LC_API int lc_contract(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                const int32_t *labels, int64_t n_c, const lc_opts *opts, int64_t *c_row_ptr,
                int32_t *c_col, int32_t *c_ew, int64_t *c_vw, int64_t cap, int64_t *c_nnz);

/* Exact objective of a clustering (Eq. 1): res->phi, res->objective,
 * res->modularity and res->n_clusters (number of distinct labels).  labels:
 * device int32[n] with values in [0, n). */
LC_API int lc_objective(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                 int64_t lambda_num, int64_t lambda_den, const int32_t *labels,
                 const lc_opts *opts, lc_result *res);

/* Allocation-free variant of lc_objective.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * when they need the objective (an application whose memory pool already
 * holds the whole GPU, or a latency-bound service that forbids
 * cudaMalloc/cudaFree after start-up because they can synchronise the
 * device).  It computes res->phi, res->objective, res->modularity and
 * res->n_clusters exactly as lc_objective does, with the same argument
 * layout (device pointers, caller-owned), and calls no cudaMalloc,
 * cudaFree or allocating routine.  Its scratch is one fixed array compiled
 * into liblc (about 36 MiB: 8 bytes plus 1 byte per vertex for
 * lc_objective_static_max_vertices() = 4,194,304 vertices, and a few
 * counters), held by every GPU on which the library is loaded until the
 * process exits.  A graph with more vertices is rejected with LC_ERR_ARG
 * and res->error_detail set to that maximum.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress), so make that
 * first call before any stream capture.  Every call shares the array and
 * clears the parts that must start at zero; calls whose work overlaps on
 * the GPU (e.g. issued on different streams without ordering) race on it.
 * The CSR is checked only as far as the sweep's reads need: row_ptr[0] = 0,
 * row_ptr[n] = nnz, every row inside [0, nnz] and column indices in [0, n),
 * else LC_ERR_ARG (symmetry, sortedness and weights are not validated).  Labels outside [0, n) give LC_ERR_ARG; inputs beyond the
 * exactness guards give LC_ERR_OVERFLOW.
 * Work is issued on opts->stream (opts may be NULL) and the call returns
 * after the result is on the host. */
LC_API int lc_objective_static(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                               int64_t lambda_num, int64_t lambda_den, const int32_t *labels,
                               const lc_opts *opts, lc_result *res);
/* Largest vertex count lc_objective_static accepts. */
LC_API int64_t lc_objective_static_max_vertices(void);

/* ---------------------------------------------------------------- checked build
 * The paper has no counterpart: these support debugging the library itself.
 * The library can be built with -DLC_DEBUG=1 (the Python binding's
 * build(debug=True), loaded when LC_DEBUG=1 is set in the environment).
 * That build checks, in every local-move, afterburner, update, objective and
 * contraction kernel, each index it follows against the array it addresses:
 * neighbour ids read from col against [0, n), cluster labels read from C and
 * from hash tables against [0, n), destinations D[v] against [0, n), coarse
 * ids against [0, n_c); hash probe sequences are bounded by their table's
 * capacity in both builds.  A failed check neither faults nor stops the
 * kernel: the index is replaced by 0, the first failure is recorded, and the
 * call returns LC_ERR_DEVICE with res->error_detail = site << 56 | index
 * (low 56 bits), site 1 column, 2 label, 3 destination, 4 probe overrun
 * (index = the vertex, -1 for a kept table's rebuild), 5 coarse id.  The
 * records are per process: calls running concurrently in the checked build
 * (server slots, several threads) may report one another's failures.  On
 * valid inputs both builds compute identical results; the checked build is
 * slower.
 *
 * lc_debug_enabled: 1 in the checked build, else 0.
 * lc_debug_selftest: checked build only (else LC_ERR_ARG): launches one
 * thread that fails one check on purpose (index 7 against bound 3, without
 * addressing memory) on `stream` (a cudaStream_t, null: the legacy default
 * stream), collects the records and returns LC_OK if exactly that failure
 * came back, with its encoded form in *detail (may be null). */
LC_API int lc_debug_enabled(void);
LC_API int lc_debug_selftest(void *stream, int64_t *detail);

#ifdef __cplusplus
}
#endif

#endif /* LC_H */
