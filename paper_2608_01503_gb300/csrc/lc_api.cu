// lc_api.cu — host driver of Louvain+ (Algorithm 1) and the C ABI of liblc.
//
// The driver issues every kernel on the caller's stream.  Per local-move
// pass nothing is read back: the best-of test (Algorithm 2) and the
// new-singleton bookkeeping run on the device.  Per level the host reads the
// bin sizes, the cluster count n_c and the coarse edge count, which size the
// launches and the coarse graph G_{l+1}.  All scratch memory comes from the
// call's provider (lc_memory.cuh: the caller's allocator or the library's
// private pool) and is sized once for G_0 and reused by every coarser level
// (Section IV-C-1, memory reuse); only coarse graphs are allocated per
// level.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lc_constraint.cuh"
#include "lc_contract.cuh"
#include "lc_leiden.cuh"
#include "lc_internal.cuh"
#include "lc_memory.cuh"
#include "lc_pass.cuh"
#include "lc_scan.cuh"
#include "lc_validate.cuh"

namespace lc {

// ------------------------------------------------------------ errors

#define LC_CK(call)                                       \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) {                              \
      fprintf(stderr, "liblc: %s failed: %s (%s:%d)\n", #call, cudaGetErrorString(e_), \
              __FILE__, __LINE__);                        \
      return e_ == cudaErrorMemoryAllocation ? LC_ERR_OOM : LC_ERR_CUDA; \
    }                                                     \
  } while (0)

#define LC_TRY(expr)        \
  do {                      \
    int rc_ = (expr);       \
    if (rc_ != LC_OK) return rc_; \
  } while (0)

// NVTX range over a phase of a call (levels, local moves, contraction,
// uncoarsening, pLeiden refinement) for timeline tools; without a tool
// attached a push / pop is a null check.
struct Phase {
  explicit Phase(const char *name) { nvtxRangePushA(name); }
  ~Phase() { nvtxRangePop(); }
  Phase(const Phase &) = delete;
  Phase &operator=(const Phase &) = delete;
};

static int launch_check() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "liblc: kernel launch failed: %s\n", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LC_ERR_OOM : LC_ERR_CUDA;
  }
  return LC_OK;
}

// ------------------------------------------------------------- device

// Once per device; several host threads (the server's slots) may get here
// together, so the flag is set only after the configuration is in place.
static void configure_device() {
  static std::mutex mtx;
  static uint64_t done_mask = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t bit = dev < 64 ? (1ull << dev) : 0;
  std::lock_guard<std::mutex> lock(mtx);
  if (done_mask & bit) return;
  configure_kernels();
  cudaGetLastError();
  done_mask |= bit;
}

// ------------------------------------------------------------ profile

struct Prof {
  bool on = false;
  cudaStream_t s = nullptr;
  struct Span {
    int cls;
    cudaEvent_t a, b;
    double bytes;
  };
  std::vector<Span> spans;
  int cur = -1;
  cudaEvent_t cur_a = nullptr;
  // events are reused across calls (per thread and device), so a span's end
  // costs one record and no event creation inside the span
  static std::vector<cudaEvent_t> &pool() {
    static thread_local std::unordered_map<int, std::vector<cudaEvent_t>> p;  // by device
    int dev = 0;
    cudaGetDevice(&dev);
    return p[dev];
  }
  static cudaEvent_t take() {
    auto &p = pool();
    if (!p.empty()) {
      cudaEvent_t e = p.back();
      p.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void begin(int cls) {
    if (!on) return;
    cur = cls;
    cur_a = take();
    cudaEventRecord(cur_a, s);
  }
  void end(double bytes) {
    if (!on) return;
    cudaEvent_t b = take();
    cudaEventRecord(b, s);
    spans.push_back({cur, cur_a, b, bytes});
  }
  void finish(lc_result *res) {
    for (auto &sp : spans) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, sp.a, sp.b) == cudaSuccess) {
        res->kernel_ms[sp.cls] += ms;
        res->kernel_bytes[sp.cls] += sp.bytes;
      }
      pool().push_back(sp.a);
      pool().push_back(sp.b);
    }
    spans.clear();
  }
  ~Prof() {
    for (auto &sp : spans) {
      cudaEventDestroy(sp.a);
      cudaEventDestroy(sp.b);
    }
  }
};

// ------------------------------------------------------------ the run

// One level G_l of a (packed) batch.  Graph g occupies the vertex range
// [vbase[g], vbase[g] + nv[g]) of the level; nv[g] = 0 when the graph has
// already finished coarsening below this level.
struct Level {
  LevelGraph g{};
  Bins bins{};
  Hubs hub{};
  int32_t *gid = nullptr;            // [n] graph of each vertex (nullptr: one graph)
  GraphParam *gp = nullptr;          // [G] device
  std::vector<int64_t> vbase, nv;    // [G] host
  std::vector<uint8_t> cont;         // [G] host: graph coarsens further from this level
  int32_t *Cd = nullptr;             // [n] dense coarse id (-1: graph finished here)
  const int32_t *B = nullptr;        // [n] constraint label (constrained coarsening), or none
};

struct Run {
  cudaStream_t s;
  lc_opts o;
  BinPlan plan = default_bin_plan();
  Method m;
  lc_result *res;  // [G]
  int G = 1;
  std::vector<long long> mu, Lam;
  std::vector<int> top;  // [G] last level of each graph
  Arena ar;
  Prof prof;
  // scratch sized for G_0
  int32_t *C = nullptr, *D = nullptr, *C_out = nullptr, *freelist = nullptr, *used = nullptr,
          *newid = nullptr, *cnt = nullptr, *scan32 = nullptr, *freepos = nullptr, *mrank = nullptr,
          *Cprev = nullptr, *dirty = nullptr, *dirty_list = nullptr, *movers = nullptr;
  int64_t *W = nullptr, *delta = nullptr, *bound = nullptr, *off = nullptr, *scan64 = nullptr;
  uint8_t *M = nullptr, *E = nullptr;
  AbRec *ab = nullptr;
  uint32_t *inL = nullptr;    // afterburner candidate bitmap
  AbWork *ab_list = nullptr;  // afterburner candidates by group, with their work records
  int2 *upd_list = nullptr;
  unsigned long long *gtab = nullptr;
  long long *gself = nullptr;
  Scalars *sc = nullptr;
  // per graph
  long long *phi_acc = nullptr, *phi_out = nullptr, *phi_trace = nullptr;
  long long *obj = nullptr;  // [4 G] objective update after a call's last pass
  long long *phi_final = nullptr;  // [G] Phi of C_out after each graph's last LocalMovePasses call
  long long *Tg = nullptr, *Vg = nullptr, *sw2g = nullptr;
  int *improved = nullptr;
  int32_t *gstart = nullptr;
  uint8_t *keep = nullptr;
  GraphStats *st = nullptr;
  std::vector<long long> hT, hV, hsw2;
  std::vector<cudaGraphExec_t> execs;  // captured passes (opts.graphs), freed with the call
  explicit Run(const lc_opts &o_) : s((cudaStream_t)o_.stream), o(o_), ar((cudaStream_t)o_.stream, o_) {}
  Run(const Run &) = delete;
  ~Run() {
    if (execs.empty()) return;
    cudaStreamSynchronize(s);  // replays finished before their graphs go
    for (cudaGraphExec_t e : execs) cudaGraphExecDestroy(e);
    cudaGetLastError();
  }
};

// A stream owned by the library to capture on (the caller's stream may be
// the legacy default stream, which cannot be captured); one per host thread
// and device.  Captured work is only recorded there and runs, as a graph, on
// the call's own stream.
static cudaStream_t capture_stream() {
  struct Streams {
    std::vector<cudaStream_t> s;
    ~Streams() {
      for (cudaStream_t x : s)
        if (x) cudaStreamDestroy(x);
    }
  };
  thread_local Streams st;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  if ((int)st.s.size() <= dev) st.s.resize(dev + 1, nullptr);
  if (!st.s[dev] && cudaStreamCreateWithFlags(&st.s[dev], cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    st.s[dev] = nullptr;
  }
  return st.s[dev];
}

static int alloc_per_graph(Run &r) {
  const int G = r.G;
  LC_TRY(r.ar.get(&r.phi_acc, G));
  LC_TRY(r.ar.get(&r.phi_out, G));
  LC_TRY(r.ar.get(&r.phi_trace, G));
  LC_TRY(r.ar.get(&r.obj, 4 * (int64_t)G));
  LC_TRY(r.ar.get(&r.phi_final, G));
  LC_CK(cudaMemsetAsync(r.phi_final, 0, 8 * (size_t)G, r.s));  // a graph with no vertices: Phi = 0
  LC_TRY(r.ar.get(&r.Tg, G));
  LC_TRY(r.ar.get(&r.Vg, G));
  LC_TRY(r.ar.get(&r.sw2g, G));
  LC_TRY(r.ar.get(&r.improved, G));
  LC_TRY(r.ar.get(&r.gstart, G));
  LC_TRY(r.ar.get(&r.keep, G));
  LC_CK(cudaMemsetAsync(r.Tg, 0, 8 * (size_t)G, r.s));
  LC_CK(cudaMemsetAsync(r.Vg, 0, 8 * (size_t)G, r.s));
  LC_CK(cudaMemsetAsync(r.sw2g, 0, 8 * (size_t)G, r.s));
  return LC_OK;
}

static int alloc_scratch(Run &r, int64_t n0, int64_t nnz0) {
  LC_TRY(r.ar.get(&r.C, n0));
  LC_TRY(r.ar.get(&r.D, n0));
  LC_TRY(r.ar.get(&r.C_out, n0));
  LC_TRY(r.ar.get(&r.freelist, n0));
  LC_TRY(r.ar.get(&r.used, n0));
  LC_TRY(r.ar.get(&r.newid, n0));
  LC_TRY(r.ar.get(&r.cnt, n0));
  LC_TRY(r.ar.get(&r.freepos, n0));
  LC_TRY(r.ar.get(&r.mrank, n0));
  LC_TRY(r.ar.get(&r.Cprev, n0));
  LC_TRY(r.ar.get(&r.movers, n0));
  if (r.o.tables == 1) {  // kept tables only
    LC_TRY(r.ar.get(&r.dirty, n0));
    LC_TRY(r.ar.get(&r.dirty_list, n0));
    LC_TRY(r.ar.get(&r.upd_list, upd_list_size(n0, nnz0)));
    LC_CK(cudaMemsetAsync(r.dirty, 0, sizeof(int32_t) * (size_t)(n0 > 0 ? n0 : 1), r.s));
  }
  const int64_t big = 2 * nnz0 > n0 + 1 ? 2 * nnz0 : n0 + 1;
  LC_TRY(r.ar.get(&r.scan32, scan_scratch(big)));
  LC_TRY(r.ar.get(&r.W, n0));
  LC_TRY(r.ar.get(&r.delta, n0));
  LC_TRY(r.ar.get(&r.ab, n0));
  LC_TRY(r.ar.get(&r.inL, (n0 + 31) / 32));
  LC_TRY(r.ar.get(&r.ab_list, n0));
  LC_TRY(r.ar.get(&r.bound, n0 + 1));
  LC_TRY(r.ar.get(&r.off, n0 + 1));
  LC_TRY(r.ar.get(&r.scan64, scan_scratch(n0 + 1)));
  LC_TRY(r.ar.get(&r.M, n0));
  LC_TRY(r.ar.get(&r.E, n0));
  LC_TRY(r.ar.get(&r.gtab, 2 * nnz0));
  if (r.G > 1) LC_TRY(r.ar.get(&r.gself, n0));
  LC_TRY(r.ar.get(&r.sc, 1));
  LC_CK(cudaMemsetAsync(r.gtab, 0, sizeof(unsigned long long) * (size_t)(2 * nnz0 > 0 ? 2 * nnz0 : 1), r.s));
  LC_CK(cudaMemsetAsync(r.sc, 0, sizeof(Scalars), r.s));
  return LC_OK;
}

// The degree bins of a call from its options (zeros take the defaults).
static int resolve_plan(const lc_opts &o, BinPlan *out) {
  BinPlan p = default_bin_plan();
  int64_t prev = 0;
  for (int k = 0; k < kBins - 1; ++k) {
    const int64_t v = o.bin_max_deg[k];
    if (v < 0 || v > kBinMaxDeg[k]) return LC_ERR_ARG;
    if (v > 0) p.max_deg[k] = v;
    if (p.max_deg[k] < prev) return LC_ERR_ARG;
    prev = p.max_deg[k];
  }
  if (o.hub_chunk != 0) {
    if (o.hub_chunk < 256 || o.hub_chunk > 65536) return LC_ERR_ARG;
    p.hub_chunk = o.hub_chunk;
  }
  for (int g = 0; g < 5; ++g) {
    const int32_t t = o.ab_threads[g];
    if (t == 0) continue;
    const bool fixed = g < 2 && t == p.ab_gs[g];  // bins 0 and 1 have one layout each
    // group 2 (degrees up to 256 by default) may also take half a warp per candidate
    if (!fixed && !(g >= 2 && (t == 32 || t == 128 || t == 512 || (g == 2 && t == 16)))) return LC_ERR_ARG;
    p.ab_gs[g] = t;
  }
  // kept tables share the shared-memory layout of the default bins (tab_cap)
  if (o.tables == 1 && !is_default_plan(p)) return LC_ERR_ARG;
  *out = p;
  return LC_OK;
}

// Bytes the allocations above, prepare() and level0() request for G_0 of a
// call on `G` graphs (kept in step with them), and those of one level's
// bins, hub plan, parameters, dense ids and coarse graph (bins_for,
// upload_params, compact_level, contract_level), for the footprint below.
static int64_t level0_scratch_bytes(int64_t n0, int64_t nnz0, int64_t G, int tables) {
  const int64_t n = n0 > 0 ? n0 : 1, big = 2 * nnz0 > n0 + 1 ? 2 * nnz0 : n0 + 1;
  int64_t b = G * (11 * 8 + 4 + 4 + 1);                     // alloc_per_graph
  b += 11 * 4 * n;                                           // C .. movers
  if (tables == 1) b += 2 * 4 * n + 8 * upd_list_size(n0, nnz0);
  b += 4 * scan_scratch(big);                                // scan32
  b += 2 * 8 * n + (int64_t)sizeof(AbRec) * n;               // W, delta, ab
  b += 4 * ((n0 + 31) / 32 + 1) + (int64_t)sizeof(AbWork) * n;  // inL, ab_list
  b += 2 * 8 * (n0 + 1) + 8 * scan_scratch(n0 + 1) + 2 * n;  // bound, off, scan64, M, E
  b += 8 * (2 * nnz0 > 0 ? 2 * nnz0 : 1);                    // gtab
  if (G > 1) b += 8 * n + 8 * (G + 1) + 4 * n;               // gself, graph_ptr, gid
  return b + (int64_t)sizeof(Scalars) + (int64_t)sizeof(GraphStats);
}
static int64_t level_bytes(int64_t n, int64_t nnz, int64_t G, const BinPlan &p) {
  const int64_t hubs = nnz / (p.hub_min() + 1) + 1, chunks = nnz / p.hub_chunk + hubs;
  return 4 * n + (int64_t)sizeof(VRec) * n + 4 * (kBins + 1) + 40 * chunks + 36 * hubs  // bins, hub plan
         + (int64_t)sizeof(GraphParam) * G                   // upload_params
         + 4 * n + (G > 1 ? 4 * n : 0)                      // Cd, next level's gid
         + 16 * (n + 1) + 8 * nnz;                          // coarse row_ptr, vw, col, ew
}

int64_t cluster_footprint(int64_t n, int64_t nnz, int count, const lc_opts &o) {
  BinPlan p;
  if (resolve_plan(o, &p) != LC_OK) p = default_bin_plan();
  // level 0 exactly, then coarse levels whose sizes sum to at most G_0's
  return level0_scratch_bytes(n, nnz, count, o.tables) + 2 * level_bytes(n, nnz, count, p) + (1 << 20);
}

// Degree bins of a level, and the chunk plan of its hub bin (rows longer
// than the last shared-memory bin are cut into chunks of the plan's hub_chunk edges).
static int bins_for(Run &r, Level &L) {
  LC_TRY(r.ar.get(&L.bins.lists, L.g.n));
  LC_TRY(r.ar.get(&L.bins.offs, kBins + 1));
  LC_TRY(r.ar.get(&L.bins.recs, L.g.n));
  build_bins(L.g, r.plan, L.bins, r.scan32, r.s);
  launch_vertex_records(L.g, L.gid, L.bins, r.s);
  int32_t h[kBins + 1];
  LC_CK(cudaMemcpyAsync(h, L.bins.offs, sizeof(h), cudaMemcpyDeviceToHost, r.s));
  LC_CK(cudaStreamSynchronize(r.s));
  finish_bins(L.bins, h);
  r.res->kernel_launches[LC_K_OTHER] += 4 * kBins + 1;
  L.hub = Hubs{};
  const int H = (int)L.bins.count[kHubBin];
  if (H > 0) {
    int64_t *rows = nullptr;
    LC_TRY(r.ar.get(&rows, 2 * H));
    launch_hub_rows(L.g.rp, L.bins.list[kHubBin], H, rows, r.s);
    r.res->kernel_launches[LC_K_OTHER] += 1;
    std::vector<int64_t> hrows(2 * (size_t)H);
    LC_CK(cudaMemcpyAsync(hrows.data(), rows, 16 * (size_t)H, cudaMemcpyDeviceToHost, r.s));
    LC_CK(cudaStreamSynchronize(r.s));
    std::vector<int32_t> hub_of, c0(H + 1);
    std::vector<int64_t> e0, e1;
    for (int k = 0; k < H; ++k) {
      c0[k] = (int32_t)hub_of.size();
      const int64_t ch = r.plan.hub_chunk;
      for (int64_t b = hrows[2 * k]; b < hrows[2 * k + 1]; b += ch) {
        hub_of.push_back(k);
        e0.push_back(b);
        e1.push_back(b + ch < hrows[2 * k + 1] ? b + ch : hrows[2 * k + 1]);
      }
    }
    const int Q = (int)hub_of.size();
    c0[H] = Q;
    int32_t *d_hub_of, *d_c0, *d_part_x;
    int64_t *d_e0, *d_e1;
    long long *d_acc, *d_part_g;
    LC_TRY(r.ar.get(&d_hub_of, Q));
    LC_TRY(r.ar.get(&d_c0, H + 1));
    LC_TRY(r.ar.get(&d_part_x, Q));
    LC_TRY(r.ar.get(&d_e0, Q));
    LC_TRY(r.ar.get(&d_e1, Q));
    LC_TRY(r.ar.get(&d_acc, H));
    LC_TRY(r.ar.get(&d_part_g, Q));
    LC_CK(cudaMemcpyAsync(d_hub_of, hub_of.data(), 4 * (size_t)Q, cudaMemcpyHostToDevice, r.s));
    LC_CK(cudaMemcpyAsync(d_c0, c0.data(), 4 * (size_t)(H + 1), cudaMemcpyHostToDevice, r.s));
    LC_CK(cudaMemcpyAsync(d_e0, e0.data(), 8 * (size_t)Q, cudaMemcpyHostToDevice, r.s));
    LC_CK(cudaMemcpyAsync(d_e1, e1.data(), 8 * (size_t)Q, cudaMemcpyHostToDevice, r.s));
    LC_CK(cudaMemsetAsync(d_acc, 0, 8 * (size_t)H, r.s));
    LC_CK(cudaStreamSynchronize(r.s));  // host vectors are released below
    L.hub.H = H;
    L.hub.Q = Q;
    L.hub.vtx = L.bins.list[kHubBin];
    L.hub.hub_of = d_hub_of;
    L.hub.e0 = d_e0;
    L.hub.e1 = d_e1;
    L.hub.c0 = d_c0;
    L.hub.acc = d_acc;
    L.hub.part_g = d_part_g;
    L.hub.part_x = d_part_x;
  }
  return launch_check();
}

// Uploads the per-graph constants of a level; active[g] selects the graphs
// whose vertices may move in the next LocalMovePasses call.
static int upload_params(Run &r, Level &L, const std::vector<uint8_t> &active) {
  if (!L.gp) LC_TRY(r.ar.get(&L.gp, r.G));
  std::vector<GraphParam> h(r.G);
  for (int g = 0; g < r.G; ++g) {
    h[g].mu = r.mu[g];
    h[g].Lam = r.Lam[g];
    h[g].vbase = (int32_t)L.vbase[g];
    h[g].active = active[g];
  }
  LC_CK(cudaMemcpyAsync(L.gp, h.data(), sizeof(GraphParam) * (size_t)r.G, cudaMemcpyHostToDevice, r.s));
  LC_CK(cudaStreamSynchronize(r.s));
  return LC_OK;
}

static PassArgs pass_args(Run &r, const Level &L) {
  PassArgs a{};
  a.g = L.g;
  a.m = r.m;
  a.gid = L.gid;
  a.gp = L.gp;
  a.G = r.G;
  a.gself = r.G > 1 ? r.gself : nullptr;
  a.phi_acc = r.phi_acc;
  a.phi_out = r.phi_out;
  a.improved = r.improved;
  a.C = r.C;
  a.W = r.W;
  a.D = r.D;
  a.delta = r.delta;
  a.ab = r.ab;
  a.M = r.M;
  a.sc = r.sc;
  a.gtab = r.gtab;
  a.hub = L.hub;
  a.Cprev = r.Cprev;
  a.dirty = r.dirty;
  a.dirty_list = r.dirty_list;
  a.obj = r.obj;
  a.hub_min = r.plan.hub_min();
  a.inL = r.inL;
  a.ab_list = r.ab_list;
  set_ab_groups(a, L.bins, r.plan);
  return a;
}

static int fill_per_graph(Run &r, long long *dst, long long value) {
  std::vector<long long> h(r.G, value);
  LC_CK(cudaMemcpyAsync(dst, h.data(), 8 * (size_t)r.G, cudaMemcpyHostToDevice, r.s));
  LC_CK(cudaStreamSynchronize(r.s));
  return LC_OK;
}

// Host copies for the optional trace callback (single-graph calls only).
static int emit_pass_event(Run &r, const Level &L, int level, int phase, int pass) {
  const int64_t n = L.g.n;
  PassArgs a = pass_args(r, L);
  a.phi_acc = r.phi_trace;
  LC_CK(cudaMemsetAsync(r.phi_trace, 0, 8 * (size_t)r.G, r.s));
  launch_objective(a, L.bins, r.s);
  launch_graph_sums(a, r.s);
  LC_TRY(launch_check());
  std::vector<int32_t> C(n > 0 ? n : 1), D(n > 0 ? n : 1);
  std::vector<uint8_t> M(n > 0 ? n : 1);
  long long phi = 0;
  Scalars sc;
  LC_CK(cudaMemcpyAsync(C.data(), r.C, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, r.s));
  LC_CK(cudaMemcpyAsync(D.data(), r.D, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, r.s));
  LC_CK(cudaMemcpyAsync(M.data(), r.M, n, cudaMemcpyDeviceToHost, r.s));
  LC_CK(cudaMemcpyAsync(&phi, r.phi_trace, 8, cudaMemcpyDeviceToHost, r.s));
  LC_CK(cudaMemcpyAsync(&sc, r.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, r.s));
  LC_CK(cudaStreamSynchronize(r.s));
  lc_event ev;
  memset(&ev, 0, sizeof(ev));
  ev.kind = LC_EV_PASS;
  ev.level = level;
  ev.phase = phase;
  ev.pass = pass;
  ev.n = n;
  ev.labels = C.data();
  ev.dest = D.data();
  ev.moved = M.data();
  ev.phi = phi;
  ev.count_L = sc.count_L;
  ev.count_M = sc.count_M;
  r.o.event_cb(r.o.event_ctx, &ev);
  return LC_OK;
}

// Records one pass of Algorithm 2 that is neither a first pass from
// singletons nor the last of its call (move step, best-of test, afterburner,
// update; the temperature comes from the device schedule) into an
// executable CUDA graph.  counts: kernels per class in one replay.
static int capture_pass(Run &r, Level &L, const PassArgs &a, const ApplyScratch &w, cudaGraphExec_t *out,
                        int64_t counts[LC_K_COUNT]) {
  *out = nullptr;
  cudaStream_t cs = capture_stream();
  if (!cs) return LC_ERR_CUDA;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return LC_ERR_CUDA;
  }
  for (int k = 0; k < LC_K_COUNT; ++k) counts[k] = 0;
  launch_pass_begin(r.sc, cs, 1);
  counts[LC_K_MOVE] += launch_move(a, L.bins, cs);
  counts[LC_K_APPLY] += launch_graph_sums(a, cs) + launch_bestof(a, r.C_out, cs);
  counts[LC_K_AFTERBURNER] += launch_afterburner(a, L.bins, cs);
  counts[LC_K_APPLY] += launch_apply(a, w, cs) + 1;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &g);
  if (e != cudaSuccess || !g) {
    cudaGetLastError();
    return LC_ERR_CUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    return LC_ERR_CUDA;
  }
  r.execs.push_back(*out);
  return LC_OK;
}

// Algorithm 2: `pass_limit` synchronous passes from r.C for the graphs with
// active[g]; leaves C_out (the best clustering seen, strict improvement) in
// r.C_out and Phi(C_out) per graph in r.phi_out.
static int local_move_passes(Run &r, Level &L, bool singleton, int level, int phase,
                             const std::vector<uint8_t> &active) {
  Phase range("lc.local_move");
  const int64_t n = L.g.n, nnz = L.g.nnz;
  LC_TRY(upload_params(r, L, active));
  PassArgs a = pass_args(r, L);
  ApplyScratch w{r.E, r.used, r.freelist, r.freepos, r.mrank, r.scan32};
  if (singleton) {
    launch_iota(r.C, n, r.s);
    launch_iota(r.C_out, n, r.s);
    LC_CK(cudaMemcpyAsync(r.W, L.g.vw, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, r.s));
    r.res->kernel_launches[LC_K_OTHER] += 2;
  } else {
    launch_cluster_weights(r.C, L.g.vw, r.W, n, r.s);
    r.res->kernel_launches[LC_K_OTHER] += 1;
  }
  LC_TRY(fill_per_graph(r, r.phi_out, singleton ? 0 : LLONG_MIN));  // Phi(singletons) = 0
  LC_CK(cudaMemsetAsync(r.phi_acc, 0, 8 * (size_t)r.G, r.s));
  // Kept tables (opts.tables = 1, Section IV-A-3): the first aggregation
  // pass of the call writes the tables of the vertices of degree above
  // kTabMinDeg out; every later pass updates them in place from the last
  // pass's movers and reads those vertices' argmax from them.  The last pass
  // clears them as it reads, so gtab is clean again when the call returns.
  const bool tables = r.o.tables == 1 && nnz > 0;
  bool kept = false;  // gtab holds tables matching C (updated by the next table pass)
  a.upd_list = tables ? r.upd_list : nullptr;
  // the final objective is updated from the last pass (see below)
  const bool incremental = r.o.pass_limit >= 1;
  // opts.graphs: the repeated passes replay one captured pass; every pass
  // then reads its temperature from the device schedule
  bool capture = r.o.graphs == 1 && !r.prof.on && !(r.o.event_cb && r.G == 1) && !tables &&
                 r.o.symmetry == 0;
  if (capture) {
    int tab[16][2];
    for (int k = 0; k < 16; ++k) {
      tab[k][0] = r.o.phi_num[k];
      tab[k][1] = r.o.phi_den[k];
    }
    LC_CK(cudaMemcpyAsync(r.sc->phi_tab, tab, sizeof(tab), cudaMemcpyHostToDevice, r.s));
    LC_CK(cudaMemsetAsync(&r.sc->pass_idx, 0, sizeof(int), r.s));
    a.phi_live = r.sc->phi_live;
  }
  cudaGraphExec_t exec = nullptr;
  int64_t exec_counts[LC_K_COUNT];
  for (int i = 1; i <= r.o.pass_limit; ++i) {
    a.phi_n = r.o.phi_num[i - 1];
    a.phi_d = r.o.phi_den[i - 1];
    const bool last = i == r.o.pass_limit;
    if (capture && !last && !(i == 1 && singleton)) {
      PassArgs ga = a;  // a repeated pass lists no movers and builds no tables
      ga.movers = nullptr;
      ga.tab_build = 0;
      if (!exec && capture_pass(r, L, ga, w, &exec, exec_counts) != LC_OK) {
        // capture is an optimisation only: the same pass, launched directly
        capture = exec != nullptr;
      }
      if (exec) {
        LC_CK(cudaGraphLaunch(exec, r.s));
        for (int k = 0; k < LC_K_COUNT; ++k) r.res->kernel_launches[k] += exec_counts[k];
        r.res->passes_total++;
        r.res->edges_local_move += nnz;
        continue;
      }
    }
    launch_pass_begin(r.sc, r.s, a.phi_live ? 1 : 0);
    a.movers = incremental && last ? r.movers : nullptr;  // listed by this pass's update step
    if (incremental && last) {
      r.prof.begin(LC_K_OBJECTIVE);
      r.res->kernel_launches[LC_K_OBJECTIVE] += launch_last_pass_enter(a, r.s);
      r.prof.end(16.0 * n);
    }
    if (i == 1 && singleton) {
      r.prof.begin(LC_K_FIRST_PASS);
      r.res->kernel_launches[LC_K_FIRST_PASS] += launch_first_pass(a, L.bins, r.s);
      r.prof.end(16.0 * nnz + 44.0 * n);
      if (incremental && last)  // Phi of the singletons, 0
        r.res->kernel_launches[LC_K_OBJECTIVE] += launch_save_phi_enter(a, r.s);
    } else {
      if (kept) {
        a.tab_build = 0;
        a.tab_reset = i == r.o.pass_limit;
        r.prof.begin(LC_K_TABLE);
        r.res->kernel_launches[LC_K_TABLE] += launch_table_pass(a, L.bins, r.s);
        // every table slot + the per-vertex reads and writes of the move step
        // (+ 40 B per updated edge, added from sc->tab_upd_edges at the end)
        r.prof.end(16.0 * nnz + 48.0 * n);
        kept = !a.tab_reset;
      } else {
        a.tab_build = tables && i < r.o.pass_limit;
        r.prof.begin(LC_K_MOVE);
        r.res->kernel_launches[LC_K_MOVE] += launch_move(a, L.bins, r.s);
        // + 8 B per distinct adjacent cluster (its W(X)), added from sc->distinct_x at the end
        r.prof.end(12.0 * nnz + 48.0 * n + (a.tab_build ? 16.0 * nnz : 0.0));
        kept = a.tab_build != 0;
        a.tab_build = 0;
      }
      r.prof.begin(LC_K_APPLY);
      r.res->kernel_launches[LC_K_APPLY] += launch_graph_sums(a, r.s);
      // Phi entering the last pass, per graph, before the best-of test resets it
      if (incremental && last) r.res->kernel_launches[LC_K_OBJECTIVE] += launch_save_phi_enter(a, r.s);
      r.res->kernel_launches[LC_K_APPLY] += launch_bestof(a, r.C_out, r.s);
      r.prof.end(8.0 * n);
    }
    r.prof.begin(LC_K_AFTERBURNER);
    if (r.o.symmetry == 0)
      r.res->kernel_launches[LC_K_AFTERBURNER] += launch_afterburner(a, L.bins, r.s);
    else  // ablations: no filter, or the minimum label heuristic in odd passes
      r.res->kernel_launches[LC_K_AFTERBURNER] +=
          launch_symmetry_ablation(a, r.o.symmetry == 2 && i % 2 == 1, r.cnt, r.s);
    r.prof.end(32.0 * n);  // + 24 B per candidate edge, added from sc->cand_edges at the end
    r.prof.begin(LC_K_APPLY);
    r.res->kernel_launches[LC_K_APPLY] += launch_apply(a, w, r.s);
    r.prof.end(14.0 * n);
    LC_TRY(launch_check());
    r.res->passes_total++;
    r.res->edges_local_move += nnz;
    if (r.o.event_cb && r.G == 1) LC_TRY(emit_pass_event(r, L, level, phase, i));
  }
  if (kept) LC_CK(cudaMemsetAsync(r.gtab, 0, 16 * (size_t)nnz, r.s));  // defensive: the last pass cleared them
  // Phi of the final state for the best-of test, updated per graph from
  // the state entering the last pass and that pass's moves
  r.prof.begin(LC_K_OBJECTIVE);
  if (incremental) {
    r.res->kernel_launches[LC_K_OBJECTIVE] += launch_final_objective(a, r.s) + launch_bestof(a, r.C_out, r.s);
    r.prof.end(17.0 * n);  // W, w(v) and M per vertex (+ 13 B per mover edge, added at the end)
  } else {
    r.res->kernel_launches[LC_K_OBJECTIVE] +=
        launch_objective(a, L.bins, r.s) + launch_graph_sums(a, r.s) + launch_bestof(a, r.C_out, r.s);
    r.prof.end(12.0 * nnz + 32.0 * n);
  }
  r.res->kernel_launches[LC_K_OTHER] += launch_keep_phi(a, r.phi_final, r.s);
  LC_TRY(launch_check());
  if (r.o.event_cb && r.G == 1) {
    std::vector<int32_t> C(n > 0 ? n : 1);
    long long phi_out = 0;
    LC_CK(cudaMemcpyAsync(C.data(), r.C_out, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, r.s));
    LC_CK(cudaMemcpyAsync(&phi_out, r.phi_out, sizeof(long long), cudaMemcpyDeviceToHost, r.s));
    LC_CK(cudaStreamSynchronize(r.s));
    lc_event ev;
    memset(&ev, 0, sizeof(ev));
    ev.kind = LC_EV_LMP;
    ev.level = level;
    ev.phase = phase;
    ev.n = n;
    ev.labels = C.data();
    ev.phi = phi_out;
    r.o.event_cb(r.o.event_ctx, &ev);
  }
  return LC_OK;
}

// The coarsening passes of a constrained level: the same passes run on G_l
// without the edges between constraint classes (lc_constraint.cu states
// why they are identical).  L keeps its full graph and bins on return.
static int constrained_passes(Run &r, Level &L, int level, const std::vector<uint8_t> &present) {
  const LevelGraph full = L.g;
  const Bins full_bins = L.bins;
  const Hubs full_hub = L.hub;
  int64_t *rp_f = nullptr;
  LC_TRY(r.ar.get(&rp_f, full.n + 1));
  r.prof.begin(LC_K_OTHER);
  launch_filter_count(full, L.B, r.cnt, r.s);
  launch_contract_rowptr(r.cnt, full.n, rp_f, r.scan64, r.s);
  int64_t nnz_f = 0;
  LC_CK(cudaMemcpyAsync(&nnz_f, rp_f + full.n, sizeof(int64_t), cudaMemcpyDeviceToHost, r.s));
  LC_CK(cudaStreamSynchronize(r.s));
  LC_TRY(launch_check());
  int32_t *col_f = nullptr, *ew_f = nullptr;
  LC_TRY(r.ar.get(&col_f, nnz_f));
  LC_TRY(r.ar.get(&ew_f, nnz_f));
  launch_filter_copy(full, L.B, rp_f, col_f, ew_f, r.s);
  r.prof.end(20.0 * full.nnz + 16.0 * full.n + 8.0 * nnz_f);
  r.res->kernel_launches[LC_K_OTHER] += 5;
  L.g = LevelGraph{full.n, nnz_f, rp_f, col_f, ew_f, full.vw};
  int rc = bins_for(r, L);
  int32_t *lists_f = L.bins.lists;
  if (rc == LC_OK) rc = local_move_passes(r, L, true, level, 0, present);
  L.g = full;
  L.bins = full_bins;
  L.hub = full_hub;
  if (rc == LC_OK) {
    r.ar.release(col_f);
    r.ar.release(ew_f);
    r.ar.release(rp_f);
    if (lists_f != full_bins.lists) r.ar.release(lists_f);
  }
  return rc;
}

// Per-graph number of labels used by C (host nc[G]); also leaves newid
// (global ascending numbering) and gstart on the device.
static int count_labels(Run &r, Level &L, const int32_t *C, std::vector<int64_t> &nc, int64_t *total) {
  const int64_t n = L.g.n;
  launch_mark_used(C, n, r.used, r.s);
  launch_number_labels(r.used, n, L.gid, L.gp, nullptr, r.newid, r.gstart, nullptr, r.scan32, r.s);
  r.res->kernel_launches[LC_K_CONTRACT] += 4;
  std::vector<int32_t> gs(r.G);
  int32_t tot = 0;
  LC_CK(cudaMemcpyAsync(gs.data(), r.gstart, 4 * (size_t)r.G, cudaMemcpyDeviceToHost, r.s));
  LC_CK(cudaMemcpyAsync(&tot, compact_total(r.scan32, n), 4, cudaMemcpyDeviceToHost, r.s));
  LC_CK(cudaStreamSynchronize(r.s));
  LC_TRY(launch_check());
  nc.assign(r.G, 0);
  int prev = -1;
  for (int g = 0; g < r.G; ++g) {
    if (L.nv[g] == 0) continue;
    if (prev >= 0) nc[prev] = gs[g] - gs[prev];
    prev = g;
  }
  if (prev >= 0) nc[prev] = tot - gs[prev];
  *total = tot;
  return LC_OK;
}

// End of a coarsening level: which graphs continue (|C_l| < |V_l|,
// Algorithm 1), their dense coarse ids L.Cd and the next level's layout.
static int compact_level(Run &r, Level &L, Level &N, int level, bool *any) {
  const int64_t n = L.g.n;
  std::vector<int64_t> nc;
  int64_t total = 0;
  r.prof.begin(LC_K_CONTRACT);
  LC_TRY(count_labels(r, L, r.C_out, nc, &total));
  L.cont.assign(r.G, 0);
  *any = false;
  for (int g = 0; g < r.G; ++g) {
    if (L.nv[g] == 0) continue;
    if (nc[g] < L.nv[g]) {
      L.cont[g] = 1;
      *any = true;
    } else {
      r.top[g] = level;
    }
  }
  if (!*any) {
    r.prof.end(24.0 * n);
    return LC_OK;
  }
  N.vbase.assign(r.G, 0);
  N.nv.assign(r.G, 0);
  int64_t base = 0;
  for (int g = 0; g < r.G; ++g) {
    if (!L.cont[g]) continue;
    N.vbase[g] = base;
    N.nv[g] = nc[g];
    base += nc[g];
  }
  N.g.n = base;
  LC_TRY(r.ar.get(&L.Cd, n));
  if (r.G > 1) LC_TRY(r.ar.get(&N.gid, N.g.n));
  LC_CK(cudaMemcpyAsync(r.keep, L.cont.data(), (size_t)r.G, cudaMemcpyHostToDevice, r.s));
  launch_number_labels(r.used, n, L.gid, L.gp, r.keep, r.newid, r.gstart, N.gid, r.scan32, r.s);
  launch_relabel(r.C_out, r.newid, L.Cd, n, L.gid, r.gstart, r.keep, 0, r.s);
  LC_CK(cudaStreamSynchronize(r.s));  // L.cont is read by the copy above
  r.prof.end(24.0 * n);
  r.res->kernel_launches[LC_K_CONTRACT] += 4;
  return launch_check();
}

// Algorithm 4 on (L.g, L.Cd) into N (whose n, vbase, nv, gid are set).
static int contract_level(Run &r, Level &L, Level &N, int level) {
  Phase range("lc.contract");
  const int64_t n_c = N.g.n;
  int64_t *rp_c = nullptr, *vw_c = nullptr;
  LC_TRY(r.ar.get(&rp_c, n_c + 1));
  LC_TRY(r.ar.get(&vw_c, n_c));
  r.prof.begin(LC_K_CONTRACT);
  launch_contract_offsets(L.g, L.Cd, n_c, r.bound, r.off, vw_c, r.scan64, r.s);
  const int ni = launch_contract_insert(L.g, L.Cd, r.off, r.gtab, r.cnt, n_c, &r.sc->error,
                                       L.bins.list, L.bins.count, L.hub, r.s);
  launch_contract_rowptr(r.cnt, n_c, rp_c, r.scan64, r.s);
  r.prof.end(16.0 * L.g.nnz + 48.0 * L.g.n);
  int64_t nnz_c = 0;
  LC_CK(cudaMemcpyAsync(&nnz_c, rp_c + n_c, sizeof(int64_t), cudaMemcpyDeviceToHost, r.s));
  LC_CK(cudaStreamSynchronize(r.s));
  LC_TRY(launch_check());
  int32_t *col_c = nullptr, *ew_c = nullptr;
  LC_TRY(r.ar.get(&col_c, nnz_c));
  LC_TRY(r.ar.get(&ew_c, nnz_c));
  r.prof.begin(LC_K_CONTRACT);
  launch_contract_compact(r.gtab, 2 * L.g.nnz, col_c, ew_c, r.scan32, r.s);
  r.prof.end(16.0 * L.g.nnz + 8.0 * nnz_c);
  r.res->kernel_launches[LC_K_CONTRACT] += 11 + ni;
  LC_TRY(launch_check());
  r.res->edges_contract += L.g.nnz;
  N.g.nnz = nnz_c;
  N.g.rp = rp_c;
  N.g.col = col_c;
  N.g.ew = ew_c;
  N.g.vw = vw_c;
  if (r.o.event_cb && r.G == 1) {
    std::vector<int64_t> h_rp(n_c + 1), h_vw(n_c > 0 ? n_c : 1);
    std::vector<int32_t> h_col(nnz_c > 0 ? nnz_c : 1), h_ew(nnz_c > 0 ? nnz_c : 1),
        h_C(L.g.n > 0 ? L.g.n : 1);
    LC_CK(cudaMemcpyAsync(h_rp.data(), rp_c, 8 * (n_c + 1), cudaMemcpyDeviceToHost, r.s));
    LC_CK(cudaMemcpyAsync(h_vw.data(), vw_c, 8 * n_c, cudaMemcpyDeviceToHost, r.s));
    LC_CK(cudaMemcpyAsync(h_col.data(), col_c, 4 * nnz_c, cudaMemcpyDeviceToHost, r.s));
    LC_CK(cudaMemcpyAsync(h_ew.data(), ew_c, 4 * nnz_c, cudaMemcpyDeviceToHost, r.s));
    LC_CK(cudaMemcpyAsync(h_C.data(), L.Cd, 4 * L.g.n, cudaMemcpyDeviceToHost, r.s));
    LC_CK(cudaStreamSynchronize(r.s));
    lc_event ev;
    memset(&ev, 0, sizeof(ev));
    ev.kind = LC_EV_CONTRACT;
    ev.level = level;
    ev.n = L.g.n;
    ev.labels = h_C.data();
    ev.cn = n_c;
    ev.cnnz = nnz_c;
    ev.c_row_ptr = h_rp.data();
    ev.c_col = h_col.data();
    ev.c_ew = h_ew.data();
    ev.c_vw = h_vw.data();
    r.o.event_cb(r.o.event_ctx, &ev);
  }
  return LC_OK;
}

// ---------------------------------------------------------- arguments

static int check_opts(const lc_opts &o) {
  if (o.pass_limit < 0 || o.pass_limit > 16) return LC_ERR_ARG;
  if (o.graphs < 0 || o.graphs > 1) return LC_ERR_ARG;
  for (int i = 0; i < o.pass_limit; ++i)
    if (o.phi_den[i] <= 0 || o.phi_num[i] < 0 || o.phi_num[i] > o.phi_den[i]) return LC_ERR_ARG;
  if (o.eps_num <= 0 || o.eps_den <= 0) return LC_ERR_ARG;
  if (o.symmetry < 0 || o.symmetry > 2) return LC_ERR_ARG;
  if (o.tables < 0 || o.tables > 1) return LC_ERR_ARG;
  if (o.scratch_limit < 0) return LC_ERR_ARG;
  if ((o.alloc == nullptr) != (o.dealloc == nullptr)) return LC_ERR_ARG;
  return LC_OK;
}

static int check_lambda(int64_t mu, int64_t Lam) {
  return (Lam <= 0 || mu < 0 || mu > Lam) ? LC_ERR_ARG : LC_OK;
}

static int check_graph_args(const lc_csr *g, const int64_t *vw, const int32_t *ew) {
  if (!g || g->n < 0 || g->n > INT32_MAX || g->nnz < 0) return LC_ERR_ARG;
  if (g->n > 0 && (!g->row_ptr || !vw)) return LC_ERR_ARG;
  if (g->nnz > 0 && (!g->col || !ew)) return LC_ERR_ARG;
  return LC_OK;
}

// Statistics, validation and the exactness guards of the header, per graph.
static int prepare(Run &r, const LevelGraph &g, const int32_t *gid, GraphStats *hst) {
  LC_TRY(r.ar.get(&r.st, 1));
  GraphStats z{};
  z.err_key = ~0ull;
  LC_CK(cudaMemcpyAsync(r.st, &z, sizeof(z), cudaMemcpyHostToDevice, r.s));
  int64_t ends[2] = {0, 0};
  LC_CK(cudaMemcpyAsync(&ends[0], g.rp, 8, cudaMemcpyDeviceToHost, r.s));
  LC_CK(cudaMemcpyAsync(&ends[1], g.rp + g.n, 8, cudaMemcpyDeviceToHost, r.s));
  LC_CK(cudaStreamSynchronize(r.s));
  if (ends[0] != 0 || ends[1] != g.nnz) return LC_ERR_ARG;
  r.prof.begin(LC_K_OTHER);
  launch_stats(g, r.o.validate, r.st, gid, r.Tg, r.Vg, r.sw2g, r.s);
  r.prof.end(16.0 * g.n + 8.0 * g.nnz);
  r.res->kernel_launches[LC_K_OTHER] += g.nnz > 0 ? 2 : 1;
  LC_CK(cudaMemcpyAsync(hst, r.st, sizeof(GraphStats), cudaMemcpyDeviceToHost, r.s));
  r.hT.assign(r.G, 0);
  r.hV.assign(r.G, 0);
  r.hsw2.assign(r.G, 0);
  if (gid) {
    LC_CK(cudaMemcpyAsync(r.hT.data(), r.Tg, 8 * (size_t)r.G, cudaMemcpyDeviceToHost, r.s));
    LC_CK(cudaMemcpyAsync(r.hV.data(), r.Vg, 8 * (size_t)r.G, cudaMemcpyDeviceToHost, r.s));
    LC_CK(cudaMemcpyAsync(r.hsw2.data(), r.sw2g, 8 * (size_t)r.G, cudaMemcpyDeviceToHost, r.s));
  }
  LC_CK(cudaStreamSynchronize(r.s));
  LC_TRY(launch_check());
  if (!gid) {
    r.hT[0] = hst->T;
    r.hV[0] = hst->V;
    r.hsw2[0] = hst->sw2;
  }
  if (r.o.validate) {
    if (hst->err_key != ~0ull) {
      r.res->error_detail = (int64_t)(hst->err_key & 0xFFFFFFFFFFull);
      return (int)(hst->err_key >> 40);
    }
    if (hst->fp1 != 0 || hst->fp2 != 0) return LC_ERR_ASYMMETRIC;
  }
  // exactness guards, per graph
  for (int k = 0; k < r.G; ++k) {
    const __int128 T = r.hT[k], V = r.hV[k];
    if (T < 0 || T >= ((__int128)1 << 31)) return LC_ERR_OVERFLOW;
    if (V < 0 || V >= ((__int128)1 << 62)) return LC_ERR_OVERFLOW;
    const __int128 B = (__int128)r.Lam[k] * T + (__int128)r.mu[k] * V * V;
    if (B >= ((__int128)1 << 60)) return LC_ERR_OVERFLOW;
    const __int128 qb = (__int128)r.m.eps_den * 2 * B / ((__int128)r.m.eps_num * r.Lam[k]);
    if (qb >= ((__int128)1 << 60)) return LC_ERR_OVERFLOW;
  }
  return LC_OK;
}

static void fill_method(Run &r) {
  r.m.eps_num = r.o.eps_num;
  r.m.eps_den = r.o.eps_den;
  r.m.seed = r.o.seed;
}

static void finish_result(Run &r, int g, lc_result *res, long long phi) {
  res->phi = phi;
  res->lambda_den = r.Lam[g];
  res->objective = (double)phi / (double)r.Lam[g];
  const long long num = phi - (r.mu[g] ? r.mu[g] * r.hsw2[g] : 0);
  res->modularity = r.hT[g] > 0 ? (double)num / ((double)r.Lam[g] * (double)r.hT[g]) : 0.0;
}

// Phi(labels) per graph through the objective kernels (labels copied to r.C).
static int objective_of(Run &r, Level &L, const int32_t *labels, std::vector<long long> &phi) {
  const int64_t n = L.g.n;
  LC_CK(cudaMemcpyAsync(r.C, labels, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, r.s));
  launch_cluster_weights(r.C, L.g.vw, r.W, n, r.s);
  PassArgs a = pass_args(r, L);
  LC_CK(cudaMemsetAsync(r.phi_acc, 0, 8 * (size_t)r.G, r.s));
  r.prof.begin(LC_K_OBJECTIVE);
  r.res->kernel_launches[LC_K_OBJECTIVE] += launch_objective(a, L.bins, r.s) + launch_graph_sums(a, r.s) + 1;
  r.prof.end(12.0 * L.g.nnz + 32.0 * n);
  phi.assign(r.G, 0);
  LC_CK(cudaMemcpyAsync(phi.data(), r.phi_acc, 8 * (size_t)r.G, cudaMemcpyDeviceToHost, r.s));
  LC_CK(cudaStreamSynchronize(r.s));
  return launch_check();
}

static int check_device_error(Run &r) {
  int err = 0;
  LC_CK(cudaMemcpyAsync(&err, &r.sc->error, sizeof(int), cudaMemcpyDeviceToHost, r.s));
  LC_CK(cudaStreamSynchronize(r.s));
#if LC_DEBUG
  // the checked build: the first failed index check of the call
  DbgRecord f{};
  if (dbg_collect(r.s, &f) > 0) {
    r.res->error_detail = ((int64_t)f.site << 56) | (f.index & ((1ll << 56) - 1));
    return LC_ERR_DEVICE;
  }
#endif
  return err ? LC_ERR_DEVICE : LC_OK;
}

// Level 0 of a call: the caller's graph, graph ids of a packed batch.
static int level0(Run &r, Level &L, const LevelGraph &g0, const std::vector<int64_t> &gptr) {
  L.g = g0;
  L.vbase.assign(r.G, 0);
  L.nv.assign(r.G, 0);
  for (int g = 0; g < r.G; ++g) {
    L.vbase[g] = gptr[g];
    L.nv[g] = gptr[g + 1] - gptr[g];
  }
  if (r.G > 1) {
    int64_t *d_gptr = nullptr;
    LC_TRY(r.ar.get(&d_gptr, r.G + 1));
    LC_TRY(r.ar.get(&L.gid, g0.n));
    LC_CK(cudaMemcpyAsync(d_gptr, gptr.data(), 8 * (size_t)(r.G + 1), cudaMemcpyHostToDevice, r.s));
    launch_graph_ids(d_gptr, r.G, L.gid, g0.n, r.s);
    LC_CK(cudaStreamSynchronize(r.s));
    r.res->kernel_launches[LC_K_OTHER] += 1;
  }
  return LC_OK;
}

// Algorithm 1 on every graph of the call; labels_out gets each graph's dense
// ids 0..k-1 (numbered within the graph).
static int cluster_impl(Run &r, const LevelGraph &g0, const std::vector<int64_t> &gptr,
                        int32_t *labels_out, const int32_t *B0 = nullptr) {
  Phase call_range("lc.cluster");
  GraphStats st{};
  LC_TRY(alloc_per_graph(r));
  std::vector<Level> lv(1);
  LC_TRY(level0(r, lv[0], g0, gptr));
  lv[0].B = B0;
  LC_TRY(prepare(r, g0, lv[0].gid, &st));
  LC_TRY(alloc_scratch(r, g0.n, g0.nnz));
  r.top.assign(r.G, 0);
  int top = 0;
  for (int l = 0;; ++l) {
    if (l >= kMaxLevels) return LC_ERR_TIMEOUT;
    Phase level_range("lc.level");
    Level &L = lv[l];
    LC_TRY(bins_for(r, L));
    std::vector<uint8_t> present(r.G);
    for (int g = 0; g < r.G; ++g) present[g] = L.nv[g] > 0;
    if (L.B)
      LC_TRY(constrained_passes(r, L, l, present));
    else
      LC_TRY(local_move_passes(r, L, true, l, 0, present));
    Level N;
    bool any = false;
    LC_TRY(compact_level(r, lv[l], N, l, &any));
    if (!any) {
      top = l;
      break;
    }
    lv.push_back(std::move(N));
    LC_TRY(contract_level(r, lv[l], lv[l + 1], l));
    if (lv[l].B) {  // coarse vertices carry their members' constraint label
      int32_t *Bc = nullptr;
      LC_TRY(r.ar.get(&Bc, lv[l + 1].g.n));
      launch_coarse_constraint(lv[l].Cd, lv[l].B, Bc, lv[l].g.n, r.s);
      r.res->kernel_launches[LC_K_OTHER] += 1;
      lv[l + 1].B = Bc;
    }
  }
  for (int g = 0; g < r.G; ++g) {
    lc_result &res = r.res[g];
    res.levels = lv[0].nv[g] > 0 ? r.top[g] + 1 : 0;
  }
  // uncoarsening; at the top level every present graph has the singleton
  // clustering its last local-move call returned
  launch_iota(r.C_out, lv[top].g.n, r.s);
  for (int l = top - 1; l >= 0; --l) {
    Phase up_range("lc.uncoarsen");
    Level &L = lv[l];
    // the level's parameters were last uploaded by its coarsening call
    launch_project(L.Cd, r.C_out, r.C, L.g.n, L.gid, L.gp, lv[l + 1].gp, r.s);
    r.res->kernel_launches[LC_K_OTHER] += 1;
    if (r.o.uncoarsen) {
      LC_TRY(local_move_passes(r, L, false, l, 1, L.cont));
    } else {
      LC_CK(cudaMemcpyAsync(r.C_out, r.C, sizeof(int32_t) * L.g.n, cudaMemcpyDeviceToDevice, r.s));
    }
  }
  // final dense labels per graph and the exact objective per graph
  Level &L0 = lv[0];
  std::vector<int64_t> nc;
  int64_t total = 0;
  LC_TRY(count_labels(r, L0, r.C_out, nc, &total));
  launch_relabel(r.C_out, r.newid, labels_out, L0.g.n, L0.gid, r.gstart, nullptr, 1, r.s);
  std::vector<long long> phi;
  if (r.o.uncoarsen && r.o.pass_limit >= 1 && !B0) {
    // each graph's final clustering is the C_out of its last LocalMovePasses
    // call, at level 0 (the uncoarsening call, or the coarsening call of a
    // graph that stopped there), whose best-of test left its exact Phi
    phi.assign(r.G, 0);
    LC_CK(cudaMemcpyAsync(phi.data(), r.phi_final, 8 * (size_t)r.G, cudaMemcpyDeviceToHost, r.s));
    LC_CK(cudaStreamSynchronize(r.s));
  } else {
    LC_TRY(objective_of(r, L0, r.C_out, phi));
  }
  LC_TRY(check_device_error(r));
  for (int g = 0; g < r.G; ++g) {
    lc_result &res = r.res[g];
    res.n_clusters = nc[g];
    if (L0.nv[g] > 0) {
      const int lev = r.top[g] + 1;
      res.passes_total = r.o.pass_limit * (lev + (r.o.uncoarsen ? lev - 1 : 0));
    }
    finish_result(r, g, &res, phi[g]);
  }
  if (r.G > 1) r.res[0].passes_total = r.o.pass_limit * (r.top[0] + 1 + (r.o.uncoarsen ? r.top[0] : 0));
  return LC_OK;
}

static lc_opts resolve_opts(const lc_opts *o) {
  lc_opts d;
  lc_default_opts(&d);
  return o ? *o : d;
}

static int begin_call(Run &r, const lc_opts *opts, lc_result *res, int G) {
  r.o = resolve_opts(opts);
  r.res = res;
  r.G = G;
  memset(res, 0, sizeof(lc_result) * (size_t)G);
  LC_TRY(check_opts(r.o));
  LC_TRY(resolve_plan(r.o, &r.plan));
  r.ar.limit = r.o.scratch_limit;
  configure_device();
  r.prof.on = r.o.profile != 0;
  r.prof.s = r.s;
  fill_method(r);
  return LC_OK;
}

static void end_call(Run &r, int rc) {
  if (rc == LC_OK && r.sc && r.o.tables == 1) {
    long long rebuilt = 0;
    if (cudaMemcpyAsync(&rebuilt, &r.sc->tab_rebuilt, sizeof(rebuilt), cudaMemcpyDeviceToHost, r.s) ==
            cudaSuccess &&
        cudaStreamSynchronize(r.s) == cudaSuccess)
      r.res->tables_rebuilt = rebuilt;
    cudaGetLastError();
  }
  if (r.prof.on) {
    cudaStreamSynchronize(r.s);
    r.prof.finish(r.res);
    long long cand = 0;  // afterburner: col, ew and the 16-byte record of each candidate edge
    if (r.sc &&
        cudaMemcpyAsync(&cand, &r.sc->cand_edges, sizeof(cand), cudaMemcpyDeviceToHost, r.s) == cudaSuccess &&
        cudaStreamSynchronize(r.s) == cudaSuccess)
      r.res->kernel_bytes[LC_K_AFTERBURNER] += 24.0 * (double)cand;
    long long upd = 0;  // kept tables: col, ew, the neighbour's row bounds, two slot updates
    if (r.sc &&
        cudaMemcpyAsync(&upd, &r.sc->tab_upd_edges, sizeof(upd), cudaMemcpyDeviceToHost, r.s) == cudaSuccess &&
        cudaStreamSynchronize(r.s) == cudaSuccess)
      r.res->kernel_bytes[LC_K_TABLE] += 40.0 * (double)upd;
    long long nx = 0;  // move step: W(X) of each distinct adjacent cluster of each vertex
    if (r.sc &&
        cudaMemcpyAsync(&nx, &r.sc->distinct_x, sizeof(nx), cudaMemcpyDeviceToHost, r.s) == cudaSuccess &&
        cudaStreamSynchronize(r.s) == cudaSuccess)
      r.res->kernel_bytes[LC_K_MOVE] += 8.0 * (double)nx;
    long long dph = 0;  // final objective: col, ew, C[u], M[u] of each mover edge
    if (r.sc &&
        cudaMemcpyAsync(&dph, &r.sc->dphi_edges, sizeof(dph), cudaMemcpyDeviceToHost, r.s) == cudaSuccess &&
        cudaStreamSynchronize(r.s) == cudaSuccess)
      r.res->kernel_bytes[LC_K_OBJECTIVE] += 13.0 * (double)dph;
    cudaGetLastError();
  }
  if (rc != LC_OK) {
    int64_t detail = r.res->error_detail;
    memset(r.res, 0, sizeof(lc_result) * (size_t)r.G);
    r.res->error_detail = detail;
  } else {
    r.res->scratch_peak_bytes = r.ar.peak;
  }
}

// Single-graph set-up shared by the step-level entry points.
static int single_graph(Run &r, const lc_csr *g, const int64_t *vw, const int32_t *ew, int64_t mu,
                        int64_t Lam, Level &L, GraphStats *st) {
  r.mu.assign(1, mu);
  r.Lam.assign(1, Lam);
  LC_TRY(alloc_per_graph(r));
  LevelGraph g0{g->n, g->nnz, g->row_ptr, g->col, ew, vw};
  std::vector<int64_t> gptr{0, g->n};
  LC_TRY(level0(r, L, g0, gptr));
  return prepare(r, g0, nullptr, st);
}

static int labels_in_range(Run &r, const int32_t *labels, int64_t n, int64_t limit) {
  launch_labels_in_range(labels, n, limit, r.st, r.s);
  GraphStats st2{};
  LC_CK(cudaMemcpyAsync(&st2, r.st, sizeof(st2), cudaMemcpyDeviceToHost, r.s));
  LC_CK(cudaStreamSynchronize(r.s));
  return st2.err_key != ~0ull ? LC_ERR_ARG : LC_OK;
}

// ----------------------------------------------------------- pLeiden

static int alloc_leiden(Run &r, int64_t n0, LeidenScratch &ls) {
  LC_TRY(r.ar.get(&ls.list, n0));
  LC_TRY(r.ar.get(&ls.list2, n0));
  LC_TRY(r.ar.get(&ls.to, n0));
  LC_TRY(r.ar.get(&ls.size, n0));
  LC_TRY(r.ar.get(&ls.H, n0));
  LC_TRY(r.ar.get(&ls.root, n0));
  LC_TRY(r.ar.get(&ls.first_bad, n0));
  LC_TRY(r.ar.get(&ls.pos, n0));
  LC_TRY(r.ar.get(&ls.f, n0));
  LC_TRY(r.ar.get(&ls.key, n0));
  LC_TRY(r.ar.get(&ls.key2, n0));
  LC_TRY(r.ar.get(&ls.WB, n0));
  LC_TRY(r.ar.get(&ls.SB, n0));
  LC_TRY(r.ar.get(&ls.Sv, n0));
  LC_TRY(r.ar.get(&ls.tv, n0));
  LC_TRY(r.ar.get(&ls.ps_w, n0));
  LC_TRY(r.ar.get(&ls.ps_t, n0));
  LC_TRY(r.ar.get(&ls.flags, n0 + 4));
  const int64_t hl = radix_hist_len(n0);
  LC_TRY(r.ar.get(&ls.hist, hl));
  LC_TRY(r.ar.get(&ls.scan64, scan_scratch(hl > n0 + 1 ? hl : n0 + 1)));
  LC_TRY(r.ar.get(&ls.scal, 4));
  LC_TRY(r.ar.get(&ls.rec, n0));
  LC_TRY(r.ar.get(&ls.krec, n0));
  return LC_OK;
}

// pLeiden (Algorithm 5) on one graph; with opts.uncoarsen, pLeiden+.  C0:
// initial clustering on the device (labels in [0, n)), or null for
// singletons.  Per level: LocalMovePasses from the level's clustering;
// LocalMoveAlt when they left Phi unchanged; stop when every cluster is a
// singleton; otherwise refine (pLeidenR with B = C_l), contract on the
// refinement and Downsample.  A refinement that merges nothing also ends
// the coarsening.
static int pleiden_impl(Run &r, const LevelGraph &g0, const int32_t *C0, int32_t *labels_out) {
  Phase call_range("lc.pleiden");
  GraphStats st{};
  LC_TRY(alloc_per_graph(r));
  std::vector<Level> lv(1);
  LC_TRY(level0(r, lv[0], g0, std::vector<int64_t>{0, g0.n}));
  LC_TRY(prepare(r, g0, nullptr, &st));
  if (C0) LC_TRY(labels_in_range(r, C0, g0.n, g0.n));  // initial labels must lie in [0, n)
  LC_TRY(alloc_scratch(r, g0.n, g0.nnz));
  LeidenScratch ls{};
  LC_TRY(alloc_leiden(r, g0.n, ls));
  int32_t *Ccur = nullptr, *Bd = nullptr, *R = nullptr;
  LC_TRY(r.ar.get(&Ccur, g0.n));
  LC_TRY(r.ar.get(&Bd, g0.n));
  LC_TRY(r.ar.get(&R, g0.n));
  if (C0)
    LC_CK(cudaMemcpyAsync(Ccur, C0, sizeof(int32_t) * (size_t)g0.n, cudaMemcpyDeviceToDevice, r.s));
  else
    launch_iota(Ccur, g0.n, r.s);
  r.top.assign(1, 0);
  const std::vector<uint8_t> present{1};
  int top = 0;
  for (int l = 0;; ++l) {
    if (l >= kMaxLevels) return LC_ERR_TIMEOUT;
    Phase level_range("lc.level");
    Level &L = lv[l];
    const int64_t n = L.g.n;
    LC_TRY(bins_for(r, L));
    LC_TRY(upload_params(r, L, present));
    std::vector<long long> phi_in;
    LC_TRY(objective_of(r, L, Ccur, phi_in));  // leaves the clustering in r.C
    LC_TRY(local_move_passes(r, L, false, l, 0, present));
    long long phi_out = 0;
    LC_CK(cudaMemcpyAsync(&phi_out, r.phi_out, sizeof(long long), cudaMemcpyDeviceToHost, r.s));
    LC_CK(cudaStreamSynchronize(r.s));
    if (phi_out == phi_in[0]) {  // LocalMoveAlt (Section V-A)
      LC_CK(cudaMemcpyAsync(r.C, r.C_out, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, r.s));
      launch_cluster_weights(r.C, L.g.vw, r.W, n, r.s);
      PassArgs a = pass_args(r, L);
      a.phi_n = 0;  // candidates: every v with g(v, D[v]) >= g(v, C[v])
      a.phi_d = 1;
      launch_pass_begin(r.sc, r.s);
      r.prof.begin(LC_K_MOVE);
      r.res->kernel_launches[LC_K_MOVE] += launch_move(a, L.bins, r.s);
      r.prof.end(12.0 * L.g.nnz + 48.0 * n);
      r.prof.begin(LC_K_ALT);
      launch_local_move_alt(L.g, L.gp, r.C, r.D, r.delta, r.W, ls, &r.sc->error, r.s);
      r.prof.end(24.0 * n);
      r.res->kernel_launches[LC_K_ALT] += 6;
      LC_CK(cudaMemcpyAsync(r.C_out, r.C, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, r.s));
      LC_TRY(launch_check());
    }
    std::vector<int64_t> nc;
    int64_t total = 0;
    LC_TRY(count_labels(r, L, r.C_out, nc, &total));
    if (total == n) {  // |C_l| = |V_l|
      top = l;
      LC_CK(cudaMemcpyAsync(Ccur, r.C_out, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, r.s));
      break;
    }
    // B = C_l with dense ids (ascending), its cluster weights, the refinement
    launch_relabel(r.C_out, r.newid, Bd, n, nullptr, r.gstart, nullptr, 0, r.s);
    launch_cluster_weights(Bd, L.g.vw, ls.WB, n, r.s);
    {
      Phase refine_range("lc.refine");
      r.prof.begin(LC_K_REFINE);
      launch_pleiden_refine(L.g, L.bins, L.gp, Bd, r.o.seed, l, R, ls, &r.sc->error, r.s);
      r.prof.end(64.0 * L.g.nnz + 200.0 * n);
    }
    r.res->kernel_launches[LC_K_REFINE] += 40;
    LC_TRY(launch_check());
    LC_CK(cudaMemcpyAsync(r.C_out, R, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, r.s));
    Level N;
    bool any = false;
    LC_TRY(compact_level(r, L, N, l, &any));
    if (!any) {  // the refinement merged nothing
      top = l;
      r.top[0] = l;
      LC_CK(cudaMemcpyAsync(Ccur, Bd, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, r.s));
      break;
    }
    lv.push_back(std::move(N));
    LC_TRY(contract_level(r, lv[l], lv[l + 1], l));
    launch_downsample(lv[l].Cd, Bd, Ccur, n, r.s);  // coarse vertex x: its members' cluster
    r.res->kernel_launches[LC_K_OTHER] += 1;
  }
  r.res->levels = top + 1;
  // uncoarsening: project, and for pLeiden+ LocalMovePasses
  LC_CK(cudaMemcpyAsync(r.C_out, Ccur, sizeof(int32_t) * lv[top].g.n, cudaMemcpyDeviceToDevice, r.s));
  for (int l = top - 1; l >= 0; --l) {
    Level &L = lv[l];
    launch_project(L.Cd, r.C_out, r.C, L.g.n, L.gid, L.gp, lv[l + 1].gp, r.s);
    r.res->kernel_launches[LC_K_OTHER] += 1;
    if (r.o.uncoarsen) {
      LC_TRY(local_move_passes(r, L, false, l, 1, present));
    } else {
      LC_CK(cudaMemcpyAsync(r.C_out, r.C, sizeof(int32_t) * L.g.n, cudaMemcpyDeviceToDevice, r.s));
    }
  }
  Level &L0 = lv[0];
  std::vector<int64_t> nc;
  int64_t total = 0;
  LC_TRY(count_labels(r, L0, r.C_out, nc, &total));
  launch_relabel(r.C_out, r.newid, labels_out, L0.g.n, nullptr, r.gstart, nullptr, 1, r.s);
  std::vector<long long> phi;
  LC_TRY(objective_of(r, L0, r.C_out, phi));
  LC_TRY(check_device_error(r));
  r.res->n_clusters = nc[0];
  finish_result(r, 0, r.res, phi[0]);
  return LC_OK;
}

}  // namespace lc

// ================================================================ C ABI

using namespace lc;

extern "C" {

void lc_default_opts(lc_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->pass_limit = 6;
  for (int i = 0; i < 16; ++i) {
    o->phi_num[i] = i < 4 ? 3 : 1;
    o->phi_den[i] = 4;
  }
  o->eps_num = 1;
  o->eps_den = 10;
  o->seed = 0;
  o->uncoarsen = 1;
  o->validate = 1;
  o->profile = 0;
  o->stream = nullptr;
  o->event_cb = nullptr;
  o->event_ctx = nullptr;
}

int lc_check_opts(const lc_opts *opts) {
  const lc_opts o = resolve_opts(opts);
  LC_TRY(check_opts(o));
  BinPlan p;
  return resolve_plan(o, &p);
}

int64_t lc_scratch_estimate(int64_t n, int64_t nnz, int32_t count, const lc_opts *opts) {
  if (n < 0 || nnz < 0 || count < 1) return -1;
  return cluster_footprint(n, nnz, count, resolve_opts(opts));
}

const char *lc_strerror(int code) {
  switch (code) {
    case LC_OK: return "ok";
    case LC_ERR_ARG: return "invalid argument";
    case LC_ERR_ASYMMETRIC: return "graph is not symmetric";
    case LC_ERR_SELF_LOOP: return "graph has a self-loop";
    case LC_ERR_DUPLICATE: return "row not strictly increasing (duplicate or unsorted)";
    case LC_ERR_WEIGHT: return "non-positive weight";
    case LC_ERR_OVERFLOW: return "exactness guard exceeded";
    case LC_ERR_OOM: return "device out of memory";
    case LC_ERR_CUDA: return "CUDA error";
    case LC_ERR_TIMEOUT: return "level limit reached";
    case LC_ERR_DEVICE: return "kernel bound violation";
    case LC_ERR_NOT_READY: return "not ready";
    default: return "unknown error";
  }
}

}  // extern "C"

namespace lc {
// lc_cluster with an optional constraint clustering B (device int32[n]).
static int cluster_single(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                          int64_t lambda_num, int64_t lambda_den, const int32_t *B,
                          const lc_opts *opts, int32_t *labels_out, lc_result *res) {
  if (!res) return LC_ERR_ARG;
  lc_opts o = resolve_opts(opts);
  Run r(o);
  int rc = begin_call(r, opts, res, 1);
  if (rc == LC_OK) rc = check_graph_args(g, vertex_w, edge_w);
  if (rc == LC_OK) rc = check_lambda(lambda_num, lambda_den);
  if (rc == LC_OK && g->n > 0 && !labels_out) rc = LC_ERR_ARG;
  if (rc == LC_OK && g->n > 0) {
    r.mu.assign(1, lambda_num);
    r.Lam.assign(1, lambda_den);
    LevelGraph g0{g->n, g->nnz, g->row_ptr, g->col, edge_w, vertex_w};
    rc = cluster_impl(r, g0, std::vector<int64_t>{0, g->n}, labels_out, B);
  } else if (rc == LC_OK) {
    res->lambda_den = lambda_den;
  }
  end_call(r, rc);
  return rc;
}
}  // namespace lc

extern "C" {

int lc_cluster(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w, int64_t lambda_num,
               int64_t lambda_den, const lc_opts *opts, int32_t *labels_out, lc_result *res) {
  return cluster_single(g, vertex_w, edge_w, lambda_num, lambda_den, nullptr, opts, labels_out, res);
}

int lc_cluster_constrained(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                           int64_t lambda_num, int64_t lambda_den, const int32_t *constraint,
                           const lc_opts *opts, int32_t *labels_out, lc_result *res) {
  if (g && g->n > 0 && !constraint) {
    if (res) memset(res, 0, sizeof(*res));
    return LC_ERR_ARG;
  }
  return cluster_single(g, vertex_w, edge_w, lambda_num, lambda_den, constraint, opts, labels_out,
                        res);
}

int lc_cluster_leiden(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w, int64_t lambda_num,
                      int64_t lambda_den, const int32_t *initial, const lc_opts *opts,
                      int32_t *labels_out, lc_result *res) {
  if (!res) return LC_ERR_ARG;
  lc_opts o = resolve_opts(opts);
  Run r(o);
  int rc = begin_call(r, opts, res, 1);
  if (rc == LC_OK) rc = check_graph_args(g, vertex_w, edge_w);
  if (rc == LC_OK) rc = check_lambda(lambda_num, lambda_den);
  if (rc == LC_OK && g->n > 0 && !labels_out) rc = LC_ERR_ARG;
  if (rc == LC_OK && g->n > 0) {
    r.mu.assign(1, lambda_num);
    r.Lam.assign(1, lambda_den);
    LevelGraph g0{g->n, g->nnz, g->row_ptr, g->col, edge_w, vertex_w};
    rc = pleiden_impl(r, g0, initial, labels_out);
  } else if (rc == LC_OK) {
    res->lambda_den = lambda_den;
  }
  end_call(r, rc);
  return rc;
}

int lc_cluster_iterated(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                        int64_t lambda_num, int64_t lambda_den, int32_t iterations,
                        const lc_opts *opts, int32_t *labels_out, lc_result *res) {
  if (!res) return LC_ERR_ARG;
  memset(res, 0, sizeof(*res));
  if (iterations < 1 || !g) return LC_ERR_ARG;
  int rc = cluster_single(g, vertex_w, edge_w, lambda_num, lambda_den, nullptr, opts, labels_out, res);
  if (rc != LC_OK || iterations == 1 || g->n == 0) return rc;
  const lc_opts o = resolve_opts(opts);
  const cudaStream_t s = (cudaStream_t)o.stream;
  int32_t *B = nullptr;
  const size_t b_bytes = sizeof(int32_t) * (size_t)g->n;
  rc = dev_alloc(o, s, b_bytes, (void **)&B);
  if (rc != LC_OK) {
    memset(res, 0, sizeof(*res));
    return rc;
  }
  lc_result total = *res;
  for (int32_t it = 1; it < iterations && rc == LC_OK; ++it) {
    if (cudaMemcpyAsync(B, labels_out, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess) {
      rc = LC_ERR_CUDA;
      break;
    }
    lc_result ri;
    rc = cluster_single(g, vertex_w, edge_w, lambda_num, lambda_den, B, opts, labels_out, &ri);
    if (rc != LC_OK) {
      total = ri;
      break;
    }
    const lc_result prev = total;
    total = ri;  // clusters, levels and objective of the last iteration
    total.scratch_peak_bytes = std::max(ri.scratch_peak_bytes, prev.scratch_peak_bytes);
    total.passes_total += prev.passes_total;
    total.edges_local_move += prev.edges_local_move;
    total.edges_contract += prev.edges_contract;
    for (int k = 0; k < LC_K_COUNT; ++k) {
      total.kernel_ms[k] += prev.kernel_ms[k];
      total.kernel_launches[k] += prev.kernel_launches[k];
      total.kernel_bytes[k] += prev.kernel_bytes[k];
    }
  }
  dev_free(o, s, B, b_bytes);
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == LC_OK) rc = LC_ERR_CUDA;
  total.scratch_peak_bytes += (int64_t)b_bytes;  // the constraint, held across the later runs
  *res = total;
  if (rc != LC_OK) {
    const int64_t detail = res->error_detail;
    memset(res, 0, sizeof(*res));
    res->error_detail = detail;
  }
  return rc;
}

int lc_cluster_batch(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w, int32_t count,
                     const int64_t *graph_ptr, const int64_t *lambda_num, const int64_t *lambda_den,
                     const lc_opts *opts, int32_t *labels_out, lc_result *res) {
  if (!res || count < 1 || !graph_ptr || !lambda_num || !lambda_den) return LC_ERR_ARG;
  lc_opts o = resolve_opts(opts);
  Run r(o);
  int rc = begin_call(r, opts, res, count);
  if (rc == LC_OK) rc = check_graph_args(g, vertex_w, edge_w);
  std::vector<int64_t> gptr(graph_ptr, graph_ptr + count + 1);
  if (rc == LC_OK) {
    if (gptr[0] != 0 || gptr[count] != g->n) rc = LC_ERR_ARG;
    for (int k = 0; rc == LC_OK && k < count; ++k)
      if (gptr[k + 1] < gptr[k] || check_lambda(lambda_num[k], lambda_den[k]) != LC_OK) rc = LC_ERR_ARG;
  }
  if (rc == LC_OK && g->n > 0 && !labels_out) rc = LC_ERR_ARG;
  if (rc == LC_OK) {
    r.mu.assign(lambda_num, lambda_num + count);
    r.Lam.assign(lambda_den, lambda_den + count);
    for (int k = 0; k < count; ++k) res[k].lambda_den = lambda_den[k];
    if (g->n > 0) {
      LevelGraph g0{g->n, g->nnz, g->row_ptr, g->col, edge_w, vertex_w};
      rc = cluster_impl(r, g0, gptr, labels_out);
    }
  }
  end_call(r, rc);
  return rc;
}

int lc_cluster_host(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                    int64_t lambda_num, int64_t lambda_den, const lc_opts *opts,
                    int32_t *labels_out, lc_result *res) {
  if (!res) return LC_ERR_ARG;
  int rc = check_graph_args(g, vertex_w, edge_w);
  if (rc != LC_OK) return rc;
  if (g->n > 0 && !labels_out) return LC_ERR_ARG;
  lc_opts o = resolve_opts(opts);
  if (check_opts(o) != LC_OK) return LC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)o.stream;
  Arena ar(s, o);
  int64_t *d_rp = nullptr, *d_vw = nullptr;
  int32_t *d_col = nullptr, *d_ew = nullptr, *d_lab = nullptr;
  const int64_t n = g->n, nnz = g->nnz;
  if ((rc = ar.get(&d_rp, n + 1)) || (rc = ar.get(&d_vw, n)) || (rc = ar.get(&d_col, nnz)) ||
      (rc = ar.get(&d_ew, nnz)) || (rc = ar.get(&d_lab, n)))
    return rc;
  if (n > 0) {
    cudaMemcpyAsync(d_rp, g->row_ptr, 8 * (n + 1), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_vw, vertex_w, 8 * n, cudaMemcpyHostToDevice, s);
  }
  if (nnz > 0) {
    cudaMemcpyAsync(d_col, g->col, 4 * nnz, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_ew, edge_w, 4 * nnz, cudaMemcpyHostToDevice, s);
  }
  if (cudaGetLastError() != cudaSuccess) return LC_ERR_CUDA;
  lc_csr dg{n, nnz, d_rp, d_col};
  rc = lc_cluster(&dg, d_vw, d_ew, lambda_num, lambda_den, &o, d_lab, res);
  if (rc == LC_OK && n > 0) {
    if (cudaMemcpyAsync(labels_out, d_lab, 4 * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = LC_ERR_CUDA;
  }
  return rc;
}

int lc_local_move(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                  int64_t lambda_num, int64_t lambda_den, const lc_opts *opts,
                  int32_t *labels_inout, int32_t singleton_start, lc_result *res) {
  if (!res) return LC_ERR_ARG;
  lc_opts o = resolve_opts(opts);
  Run r(o);
  int rc = begin_call(r, opts, res, 1);
  if (rc == LC_OK) rc = check_graph_args(g, vertex_w, edge_w);
  if (rc == LC_OK) rc = check_lambda(lambda_num, lambda_den);
  if (rc == LC_OK && g->n > 0 && !labels_inout) rc = LC_ERR_ARG;
  if (rc == LC_OK && g->n > 0) {
    Level L;
    GraphStats st{};
    rc = single_graph(r, g, vertex_w, edge_w, lambda_num, lambda_den, L, &st);
    if (rc == LC_OK) rc = labels_in_range(r, labels_inout, g->n, g->n);
    if (rc == LC_OK) rc = alloc_scratch(r, g->n, g->nnz);
    if (rc == LC_OK) rc = bins_for(r, L);
    if (rc == LC_OK) {
      cudaMemcpyAsync(r.C, labels_inout, 4 * g->n, cudaMemcpyDeviceToDevice, r.s);
      rc = local_move_passes(r, L, singleton_start != 0, 0, singleton_start ? 0 : 1,
                             std::vector<uint8_t>{1});
    }
    if (rc == LC_OK) {
      cudaMemcpyAsync(labels_inout, r.C_out, 4 * g->n, cudaMemcpyDeviceToDevice, r.s);
      long long phi = 0;
      std::vector<int64_t> nc;
      int64_t total = 0;
      if (cudaMemcpyAsync(&phi, r.phi_out, 8, cudaMemcpyDeviceToHost, r.s) != cudaSuccess)
        rc = LC_ERR_CUDA;
      if (rc == LC_OK) rc = count_labels(r, L, labels_inout, nc, &total);
      if (rc == LC_OK) rc = check_device_error(r);
      if (rc == LC_OK) {
        res->n_clusters = total;
        res->levels = 1;
        finish_result(r, 0, res, phi);
      }
    }
  }
  end_call(r, rc);
  return rc;
}

int lc_contract(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                const int32_t *labels, int64_t n_c, const lc_opts *opts, int64_t *c_row_ptr,
                int32_t *c_col, int32_t *c_ew, int64_t *c_vw, int64_t cap, int64_t *c_nnz) {
  int rc = check_graph_args(g, vertex_w, edge_w);
  if (rc != LC_OK) return rc;
  if (n_c < 0 || n_c > g->n || !c_nnz || (g->n > 0 && (!labels || !c_row_ptr || !c_vw)) ||
      cap < 0 || (cap > 0 && (!c_col || !c_ew)))
    return LC_ERR_ARG;
  if (g->n > 0 && n_c == 0) return LC_ERR_ARG;
  lc_result tmp;
  lc_opts o = resolve_opts(opts);
  Run r(o);
  rc = begin_call(r, opts, &tmp, 1);
  if (rc != LC_OK) return rc;
  *c_nnz = 0;
  if (g->n == 0) {
    if (c_row_ptr) cudaMemsetAsync(c_row_ptr, 0, 8, r.s);
    return cudaStreamSynchronize(r.s) == cudaSuccess ? LC_OK : LC_ERR_CUDA;
  }
  Level L;
  GraphStats st{};
  rc = single_graph(r, g, vertex_w, edge_w, 0, 1, L, &st);
  if (rc == LC_OK) rc = labels_in_range(r, labels, g->n, n_c);
  if (rc == LC_OK) rc = alloc_scratch(r, g->n, g->nnz);
  if (rc == LC_OK) rc = bins_for(r, L);
  if (rc == LC_OK) {
    L.Cd = const_cast<int32_t *>(labels);
    launch_contract_offsets(L.g, L.Cd, n_c, r.bound, r.off, c_vw, r.scan64, r.s);
    launch_contract_insert(L.g, L.Cd, r.off, r.gtab, r.cnt, n_c, &r.sc->error, L.bins.list,
                           L.bins.count, L.hub, r.s);
    launch_contract_rowptr(r.cnt, n_c, c_row_ptr, r.scan64, r.s);
    int64_t nnz_c = 0;
    if (cudaMemcpyAsync(&nnz_c, c_row_ptr + n_c, 8, cudaMemcpyDeviceToHost, r.s) != cudaSuccess ||
        cudaStreamSynchronize(r.s) != cudaSuccess)
      rc = LC_ERR_CUDA;
    if (rc == LC_OK && nnz_c > cap) {
      rc = LC_ERR_ARG;
      r.res->error_detail = nnz_c;
    }
    if (rc == LC_OK) {
      launch_contract_compact(r.gtab, 2 * g->nnz, c_col, c_ew, r.scan32, r.s);
      rc = launch_check();
    }
    if (rc == LC_OK) rc = check_device_error(r);
    if (rc == LC_OK) *c_nnz = nnz_c;
  }
  end_call(r, rc);
  return rc;
}

int lc_objective(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                 int64_t lambda_num, int64_t lambda_den, const int32_t *labels,
                 const lc_opts *opts, lc_result *res) {
  if (!res) return LC_ERR_ARG;
  lc_opts o = resolve_opts(opts);
  Run r(o);
  int rc = begin_call(r, opts, res, 1);
  if (rc == LC_OK) rc = check_graph_args(g, vertex_w, edge_w);
  if (rc == LC_OK) rc = check_lambda(lambda_num, lambda_den);
  if (rc == LC_OK && g->n > 0 && !labels) rc = LC_ERR_ARG;
  if (rc == LC_OK && g->n > 0) {
    Level L;
    GraphStats st{};
    rc = single_graph(r, g, vertex_w, edge_w, lambda_num, lambda_den, L, &st);
    if (rc == LC_OK) rc = labels_in_range(r, labels, g->n, g->n);
    if (rc == LC_OK) rc = alloc_scratch(r, g->n, 0);
    if (rc == LC_OK) rc = bins_for(r, L);
    if (rc == LC_OK) rc = upload_params(r, L, std::vector<uint8_t>{1});
    std::vector<long long> phi;
    if (rc == LC_OK) rc = objective_of(r, L, labels, phi);
    std::vector<int64_t> nc;
    int64_t total = 0;
    if (rc == LC_OK) rc = count_labels(r, L, labels, nc, &total);
    if (rc == LC_OK) {
      res->n_clusters = total;
      res->levels = 1;
      finish_result(r, 0, res, phi[0]);
    }
  } else if (rc == LC_OK) {
    res->lambda_den = lambda_den;
  }
  end_call(r, rc);
  return rc;
}

}  // extern "C"
