// lc_server.cu — a clustering service over lc_cluster_batch.
//
// Requests (host CSR graphs) are queued in arrival order.  A fixed number of
// slots, each a worker thread with its own CUDA stream, take work: when a
// slot is free it admits queued jobs from the head of the queue while their
// estimated device footprint fits in the memory budget still unclaimed (and
// up to max_batch jobs), packs them into one CSR and clusters them with one
// lc_cluster_batch call, so their local-move sweeps share launches.  Slots
// run concurrently, so requests arriving while others are on the GPU are
// admitted as soon as a slot and memory free up, and their work overlaps on
// the device.  Each job's result is what lc_cluster returns for it alone.
//
// A job's footprint is its packed input plus the clustering's scratch as
// estimated by lc::cluster_footprint (the driver's own allocation sizes).
// An admission's clustering runs with its reserved scratch as the call's
// scratch limit, so admitted work never holds more than the budget.  A run
// whose levels shrink too slowly for the estimate stops with LC_ERR_OOM;
// its jobs then go back to the head of the queue with twice the estimate
// and wait for memory (a job larger than the whole budget runs alone, with
// no limit), so callers only see LC_ERR_OOM when the device itself is out.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/lc.h"
#include "lc_memory.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  int64_t id = 0;
  int64_t n = 0, nnz = 0;
  std::vector<int64_t> rp, vw;
  std::vector<int32_t> col, ew;
  int64_t mu = 0, Lam = 1;
  int64_t scratch = 0;    // reserved clustering scratch (grows on retry)
  int64_t footprint = 0;  // input + scratch
  int state = 0;  // 0 queued, 1 running, 2 done
  int rc = LC_OK;
  std::vector<int32_t> labels;
  lc_result res{};
  Clock::time_point t_submit, t_done;
};

}  // namespace

struct lc_server {
  lc_server_config cfg{};
  int device = 0;
  int64_t budget = 0, claimed = 0;
  int64_t next_id = 1;
  bool stop = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int64_t> queue;
  std::unordered_map<int64_t, Job> jobs;
  std::vector<std::thread> workers;
};

namespace {

// Device bytes of a job's packed input: row pointers, vertex weights,
// columns, edge weights and labels (cluster_packed's arena), plus room for
// the provider's rounding of five blocks.
int64_t input_bytes(int64_t n, int64_t nnz) { return 8 * (n + 1) + 8 * n + 8 * nnz + 4 * n + 5 * 512; }

template <typename T>
__global__ void k_add_offset(T *__restrict__ a, int64_t count, T add) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] += add;
}

template <typename T>
void add_offset(T *a, int64_t count, T add, cudaStream_t st) {
  if (count <= 0 || add == 0) return;
  int64_t b = (count + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  k_add_offset<T><<<(unsigned)b, 256, 0, st>>>(a, count, add);
}

// Packs jobs into one CSR on the device (each job copied to its offset,
// then shifted to global ids) and clusters them in one batched call.
// labels (host, the packed vertex range) and res[k] are filled on success.
// scratch_limit: the clustering's scratch limit (0: none).
int cluster_packed(lc_server *s, cudaStream_t st, Job *const *jobs, int count, int64_t scratch_limit,
                   std::vector<int32_t> &labels, std::vector<int64_t> &gptr, lc_result *res) {
  std::vector<int64_t> eptr(count + 1, 0), lam_num(count), lam_den(count);
  gptr.assign(count + 1, 0);
  for (int k = 0; k < count; ++k) {
    gptr[k + 1] = gptr[k] + jobs[k]->n;
    eptr[k + 1] = eptr[k] + jobs[k]->nnz;
    lam_num[k] = jobs[k]->mu;
    lam_den[k] = jobs[k]->Lam;
  }
  const int64_t n = gptr[count], nnz = eptr[count];
  labels.assign(n > 0 ? n : 1, 0);
  int64_t *d_rp = nullptr, *d_vw = nullptr;
  int32_t *d_col = nullptr, *d_ew = nullptr, *d_lab = nullptr;
  lc::Arena ar(st, s->cfg.opts);
  int rc = ar.get(&d_rp, n + 1);
  if (rc == LC_OK) rc = ar.get(&d_vw, n);
  if (rc == LC_OK) rc = ar.get(&d_col, nnz);
  if (rc == LC_OK) rc = ar.get(&d_ew, nnz);
  if (rc == LC_OK) rc = ar.get(&d_lab, n);
  if (rc == LC_OK) {
    for (int k = 0; k < count; ++k) {
      const Job &j = *jobs[k];
      if (j.n > 0) {
        cudaMemcpyAsync(d_rp + gptr[k], j.rp.data(), 8 * j.n, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_vw + gptr[k], j.vw.data(), 8 * j.n, cudaMemcpyHostToDevice, st);
        add_offset<int64_t>(d_rp + gptr[k], j.n, eptr[k], st);
      }
      if (j.nnz > 0) {
        cudaMemcpyAsync(d_col + eptr[k], j.col.data(), 4 * j.nnz, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_ew + eptr[k], j.ew.data(), 4 * j.nnz, cudaMemcpyHostToDevice, st);
        add_offset<int32_t>(d_col + eptr[k], j.nnz, (int32_t)gptr[k], st);
      }
    }
    cudaMemcpyAsync(d_rp + n, &eptr[count], 8, cudaMemcpyHostToDevice, st);
    lc_opts o = s->cfg.opts;
    o.stream = st;
    o.event_cb = nullptr;
    o.profile = 0;
    o.scratch_limit = scratch_limit;
    lc_csr g{n, nnz, d_rp, d_col};
    if (cudaGetLastError() != cudaSuccess) rc = LC_ERR_CUDA;
    if (rc == LC_OK)
      rc = lc_cluster_batch(&g, d_vw, d_ew, count, gptr.data(), lam_num.data(), lam_den.data(), &o,
                            d_lab, res);
    if (rc == LC_OK && n > 0) {
      if (cudaMemcpyAsync(labels.data(), d_lab, 4 * n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = LC_ERR_CUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == LC_OK) rc = LC_ERR_CUDA;
  }
  return rc;  // the arena returns the input buffers in stream order
}

// Clusters an admission.  If the batched call fails (one request breaks a
// precondition or a guard), every job is run alone so that only the
// offending ones report an error.
// limited: the admission fits the budget, so its scratch is limited to
// what it reserved.
void run_batch(lc_server *s, cudaStream_t st, std::vector<Job *> &batch, bool limited) {
  const int count = (int)batch.size();
  std::vector<int32_t> labels;
  std::vector<int64_t> gptr;
  std::vector<lc_result> res(count);
  std::vector<int> rcs(count, LC_OK);
  std::vector<std::vector<int32_t>> own(count);
  int64_t reserved = 0;
  for (Job *j : batch) reserved += j->scratch;
  const int rc = cluster_packed(s, st, batch.data(), count, limited ? reserved : 0, labels, gptr, res.data());
  if (rc == LC_ERR_OOM && limited) {
    // the estimate was short: back to the head of the queue, in order, with
    // twice the reservation, to wait for memory
    std::lock_guard<std::mutex> lock(s->mu);
    for (int k = count - 1; k >= 0; --k) {
      Job &j = *batch[k];
      s->claimed -= j.footprint;
      j.scratch *= 2;
      j.footprint = input_bytes(j.n, j.nnz) + j.scratch;
      j.state = 0;
      s->queue.push_front(j.id);
    }
    s->cv_work.notify_all();
    return;
  }
  if (rc == LC_OK) {
    for (int k = 0; k < count; ++k) own[k].assign(labels.begin() + gptr[k], labels.begin() + gptr[k + 1]);
  } else if (count == 1) {
    rcs[0] = rc;
  } else {
    for (int k = 0; k < count; ++k) {
      rcs[k] = cluster_packed(s, st, &batch[k], 1, limited ? batch[k]->scratch : 0, labels, gptr, &res[k]);
      if (rcs[k] == LC_OK) own[k].assign(labels.begin(), labels.begin() + batch[k]->n);
    }
  }
  const auto now = Clock::now();
  std::lock_guard<std::mutex> lock(s->mu);
  for (int k = 0; k < count; ++k) {
    Job &j = *batch[k];
    j.rc = rcs[k];
    j.res = res[k];
    if (rcs[k] == LC_OK) j.labels.swap(own[k]);
    j.state = 2;
    j.t_done = now;
    s->claimed -= j.footprint;
    // the job's input copies are no longer needed
    std::vector<int64_t>().swap(j.rp);
    std::vector<int64_t>().swap(j.vw);
    std::vector<int32_t>().swap(j.col);
    std::vector<int32_t>().swap(j.ew);
  }
  s->cv_done.notify_all();
  s->cv_work.notify_all();
}

void worker(lc_server *s) {
  cudaSetDevice(s->device);
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    std::vector<Job *> batch;
    bool limited = true;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      for (;;) {
        if (s->stop && s->queue.empty()) break;
        if (!s->queue.empty()) {
          // admit from the head while the footprint fits; a job larger than
          // the whole budget runs alone once nothing else holds memory
          int64_t add = 0;
          for (int64_t id : s->queue) {
            Job &j = s->jobs[id];
            if ((int)batch.size() >= s->cfg.max_batch) break;
            const bool fits = s->claimed + add + j.footprint <= s->budget;
            const bool alone = batch.empty() && s->claimed == 0;
            if (!fits && !alone) break;
            batch.push_back(&j);
            add += j.footprint;
            if (!fits) {
              limited = false;
              break;
            }
          }
          if (!batch.empty()) {
            for (size_t k = 0; k < batch.size(); ++k) {
              s->queue.pop_front();
              batch[k]->state = 1;
            }
            s->claimed += add;
            break;
          }
        }
        s->cv_work.wait(lock);
      }
    }
    if (batch.empty()) break;
    run_batch(s, st, batch, limited);
  }
  cudaStreamDestroy(st);
}

int finish_job(lc_server *s, Job &j, int32_t *labels_out, lc_result *res, double *latency_s) {
  if (j.rc == LC_OK && labels_out && j.n > 0) memcpy(labels_out, j.labels.data(), 4 * (size_t)j.n);
  if (res) *res = j.res;  // on error: zero but for error_detail
  if (latency_s) *latency_s = std::chrono::duration<double>(j.t_done - j.t_submit).count();
  const int rc = j.rc;
  s->jobs.erase(j.id);
  return rc;
}

}  // namespace

extern "C" {

LC_API void lc_server_default_config(lc_server_config *c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->slots = 4;
  c->max_batch = 64;
  c->hbm_budget = 0;
  lc_default_opts(&c->opts);
}

LC_API int lc_server_create(const lc_server_config *cfg, lc_server **out) {
  if (!out) return LC_ERR_ARG;
  *out = nullptr;
  lc_server_config c;
  lc_server_default_config(&c);
  if (cfg) c = *cfg;
  if (c.slots < 1 || c.slots > 64 || c.max_batch < 1 || c.hbm_budget < 0) return LC_ERR_ARG;
  if ((c.opts.alloc == nullptr) != (c.opts.dealloc == nullptr)) return LC_ERR_ARG;
  lc_server *s = new lc_server();
  s->cfg = c;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return LC_ERR_CUDA;
  }
  if (c.hbm_budget == 0) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      delete s;
      return LC_ERR_CUDA;
    }
    s->budget = (int64_t)(free_b / 2);
  } else {
    s->budget = c.hbm_budget;
  }
  for (int k = 0; k < c.slots; ++k) s->workers.emplace_back(worker, s);
  *out = s;
  return LC_OK;
}

LC_API int lc_server_submit(lc_server *s, const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                     int64_t lambda_num, int64_t lambda_den, int64_t *job_id) {
  if (!s || !g || !job_id || g->n < 0 || g->nnz < 0 || g->n > INT32_MAX) return LC_ERR_ARG;
  if ((g->n > 0 && (!g->row_ptr || !vertex_w)) || (g->nnz > 0 && (!g->col || !edge_w)))
    return LC_ERR_ARG;
  if (lambda_den <= 0 || lambda_num < 0 || lambda_num > lambda_den) return LC_ERR_ARG;
  if (g->row_ptr && (g->row_ptr[0] != 0 || g->row_ptr[g->n] != g->nnz)) return LC_ERR_ARG;
  Job j;
  j.t_submit = Clock::now();  // latency includes the copy below
  j.n = g->n;
  j.nnz = g->nnz;
  if (g->row_ptr)
    j.rp.assign(g->row_ptr, g->row_ptr + g->n + 1);
  else
    j.rp.assign(1, 0);
  if (g->n > 0) j.vw.assign(vertex_w, vertex_w + g->n);
  if (g->nnz > 0) {
    j.col.assign(g->col, g->col + g->nnz);
    j.ew.assign(edge_w, edge_w + g->nnz);
  }
  j.mu = lambda_num;
  j.Lam = lambda_den;
  j.scratch = lc::cluster_footprint(g->n, g->nnz, 1, s->cfg.opts);
  j.footprint = input_bytes(g->n, g->nnz) + j.scratch;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return LC_ERR_ARG;
    j.id = s->next_id++;
    *job_id = j.id;
    s->jobs.emplace(j.id, std::move(j));
    s->queue.push_back(*job_id);
  }
  s->cv_work.notify_all();
  return LC_OK;
}

LC_API int lc_server_poll(lc_server *s, int64_t job_id, int32_t *labels_out, lc_result *res,
                   double *latency_s) {
  if (!s) return LC_ERR_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return LC_ERR_ARG;
  if (it->second.state != 2) return LC_ERR_NOT_READY;
  return finish_job(s, it->second, labels_out, res, latency_s);
}

LC_API int lc_server_wait(lc_server *s, int64_t job_id, int32_t *labels_out, lc_result *res,
                   double *latency_s) {
  if (!s) return LC_ERR_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  for (;;) {
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return LC_ERR_ARG;
    if (it->second.state == 2) return finish_job(s, it->second, labels_out, res, latency_s);
    s->cv_done.wait(lock);
  }
}

LC_API int lc_server_cancel(lc_server *s, int64_t job_id) {
  if (!s) return LC_ERR_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return LC_ERR_ARG;
  if (it->second.state != 0) return LC_ERR_NOT_READY;
  for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
    if (*q == job_id) {
      s->queue.erase(q);
      break;
    }
  s->jobs.erase(it);
  s->cv_work.notify_all();  // the head of the queue may have changed
  return LC_OK;
}

LC_API int lc_server_destroy(lc_server *s) {
  if (!s) return LC_ERR_ARG;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto &t : s->workers) t.join();
  delete s;
  return LC_OK;
}

}  // extern "C"
