// lc_tune.cu — lc_autotune: picks the launch settings of the local-move
// and contraction kernels by timing them on the caller's own workload.
//
// The paper splits vertices into degree buckets (Section IV-C-2) but leaves
// the thresholds open.  Here they are runtime options (lc_opts.bin_max_deg,
// hub_chunk) together with the CUDA-graph replay of repeated passes
// (lc_opts.graphs); none of them changes a result, only which kernel handles
// a vertex and how the work is launched.  The tuner walks the settings one
// dimension at a time (coordinate descent from the defaults), times each
// candidate with CUDA events on the call's stream (median of `repeats`
// runs after one untimed run), checks that its labels equal those of the
// defaults, and keeps a change only if it is faster.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/lc.h"
#include "lc_memory.cuh"

namespace {

struct Workload {
  const lc_csr *g;
  const int64_t *vw;
  const int32_t *ew;
  int32_t count;
  const int64_t *gptr;
  const int64_t *mu, *Lam;
  int32_t *labels;  // device scratch for the candidate's labels
  cudaStream_t s;
};

int run_once(const Workload &w, const lc_opts &o, std::vector<lc_result> &res) {
  if (w.count == 1)
    return lc_cluster(w.g, w.vw, w.ew, w.mu[0], w.Lam[0], &o, w.labels, res.data());
  return lc_cluster_batch(w.g, w.vw, w.ew, w.count, w.gptr, w.mu, w.Lam, &o, w.labels, res.data());
}

// Median milliseconds of `repeats` timed runs (after one untimed run), and
// the labels of the last run.
int time_setting(const Workload &w, const lc_opts &o, int repeats, double *ms,
                 std::vector<int32_t> &labels) {
  std::vector<lc_result> res(w.count);
  int rc = run_once(w, o, res);
  if (rc != LC_OK) return rc;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return LC_ERR_CUDA;
  std::vector<double> t;
  for (int k = 0; k < repeats && rc == LC_OK; ++k) {
    cudaEventRecord(a, w.s);
    rc = run_once(w, o, res);
    cudaEventRecord(b, w.s);
    float m = 0.f;
    if (rc == LC_OK && (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&m, a, b) != cudaSuccess))
      rc = LC_ERR_CUDA;
    t.push_back(m);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc != LC_OK) return rc;
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  labels.resize(w.g->n > 0 ? w.g->n : 1);
  if (w.g->n > 0 &&
      (cudaMemcpyAsync(labels.data(), w.labels, 4 * (size_t)w.g->n, cudaMemcpyDeviceToHost, w.s) != cudaSuccess ||
       cudaStreamSynchronize(w.s) != cudaSuccess))
    return LC_ERR_CUDA;
  return LC_OK;
}

const int kDefaultMax[9] = {8, 16, 32, 128, 256, 512, 1024, 2048, 4096};
const int kDefaultAb[5] = {1, 16, 32, 128, 512};

}  // namespace

extern "C" LC_API int lc_autotune(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                                  int32_t count, const int64_t *graph_ptr, const int64_t *lambda_num,
                                  const int64_t *lambda_den, const lc_opts *opts, int32_t repeats,
                                  lc_tuning *out) {
  if (!g || !out || count < 1 || !lambda_num || !lambda_den || (count > 1 && !graph_ptr) || repeats < 1)
    return LC_ERR_ARG;
  memset(out, 0, sizeof(*out));
  lc_opts base;
  lc_default_opts(&base);
  if (opts) base = *opts;
  base.profile = 0;
  base.event_cb = nullptr;
  if (base.tables == 1) return LC_ERR_ARG;  // kept tables need the default bins
  const cudaStream_t s = (cudaStream_t)base.stream;
  int32_t *labels = nullptr;
  const size_t lab_bytes = 4 * (size_t)(g->n > 0 ? g->n : 1);
  int rc0 = lc::dev_alloc(base, s, lab_bytes, (void **)&labels);
  if (rc0 != LC_OK) return rc0;
  Workload w{g, vertex_w, edge_w, count, graph_ptr, lambda_num, lambda_den, labels, s};

  // the current setting: the defaults (or what the caller passed)
  lc_opts cur = base;
  for (int k = 0; k < 9; ++k)
    if (cur.bin_max_deg[k] == 0) cur.bin_max_deg[k] = kDefaultMax[k];
  if (cur.hub_chunk == 0) cur.hub_chunk = 2048;
  std::vector<int32_t> ref, lab;
  double best = 0;
  int rc = time_setting(w, cur, repeats, &best, ref);
  out->ms_default = best;
  out->trials = 1;

  // a candidate replaces the current setting if it is faster and exact
  auto try_setting = [&](const lc_opts &cand) -> int {
    double ms = 0;
    const int r = time_setting(w, cand, repeats, &ms, lab);
    out->trials++;
    if (r == LC_ERR_ARG) return LC_OK;  // not a valid plan here: skip it
    if (r != LC_OK) return r;
    if (lab != ref) return LC_ERR_DEVICE;  // a setting changed a result: a library fault
    if (ms < best) {
      best = ms;
      cur = cand;
    }
    return LC_OK;
  };

  // 1. where the hubs start: above 4096 (default), 2048 or 1024
  for (int hub : {2048, 1024}) {
    if (rc != LC_OK) break;
    lc_opts c = cur;
    for (int k = 0; k < 9; ++k) c.bin_max_deg[k] = std::min(c.bin_max_deg[k], hub);
    rc = try_setting(c);
  }
  // 2. hub chunk length
  for (int ch : {1024, 4096, 8192}) {
    if (rc != LC_OK) break;
    lc_opts c = cur;
    c.hub_chunk = ch;
    rc = try_setting(c);
  }
  // 3. the lane / warp / block boundaries below the hubs, each moved down
  //    to half of its default (the neighbouring, larger bin takes the rest)
  for (int k : {2, 3, 4, 5, 6}) {
    if (rc != LC_OK) break;
    lc_opts c = cur;
    const int lo = k > 0 ? c.bin_max_deg[k - 1] : 0;
    const int v = std::max(lo, kDefaultMax[k] / 2);
    if (v >= c.bin_max_deg[k] || c.bin_max_deg[k + 1] < v) continue;
    c.bin_max_deg[k] = v;
    rc = try_setting(c);
  }
  // 4. threads per candidate in the afterburner's wide groups (group 2:
  //    half a warp or a warp)
  for (int g : {2, 3, 4}) {
    for (int t : {16, 32, 128, 512}) {
      if (g == 2 && t > 32) continue;
      if (g > 2 && t == 16) continue;
      if (rc != LC_OK) break;
      lc_opts c = cur;
      if ((c.ab_threads[g] ? c.ab_threads[g] : kDefaultAb[g]) == t) continue;
      c.ab_threads[g] = t;
      rc = try_setting(c);
    }
  }
  // 5. CUDA-graph replay of the repeated passes
  if (rc == LC_OK) {
    lc_opts c = cur;
    c.graphs = 1;
    rc = try_setting(c);
  }
  lc::dev_free(base, s, labels, lab_bytes);
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == LC_OK) rc = LC_ERR_CUDA;
  if (rc != LC_OK) return rc;
  for (int k = 0; k < 9; ++k) out->bin_max_deg[k] = cur.bin_max_deg[k];
  for (int k = 0; k < 5; ++k) out->ab_threads[k] = cur.ab_threads[k] ? cur.ab_threads[k] : kDefaultAb[k];
  out->hub_chunk = cur.hub_chunk;
  out->graphs = cur.graphs;
  out->ms_best = best;
  return LC_OK;
}
