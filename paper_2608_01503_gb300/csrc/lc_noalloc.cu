// lc_noalloc.cu — lc_objective_static: the exact LambdaCC objective of a
// clustering computed without allocating any device memory.
//
// Why it exists: some callers cannot allocate device memory at the moment
// they need an objective value.  Examples are applications whose own memory
// pool has already reserved all of the GPU's memory, and latency-sensitive
// services that forbid cudaMalloc/cudaFree after start-up because those
// calls can synchronise the device and stall unrelated streams.  Such callers
// pass their inputs and read the result back; the scratch this computation
// needs lives in one fixed array compiled into the library.
//
// The scratch array below is a file-scope __device__ array: every GPU on
// which this library's code is loaded holds it until the process exits.
// Host code cannot use the symbol's name as a device pointer, so the device
// address is fetched once per device with cudaGetSymbolAddress and passed to
// the kernels.  All calls share the array and it keeps the previous call's
// contents: each call clears what must start at zero, and two calls whose
// work overlaps on the GPU (e.g. on different streams) race on it.
#include <cuda_runtime.h>

#include <climits>
#include <cstring>
#include <mutex>

#include "../../include/lc.h"

namespace {

// Largest graph the allocation-free path accepts (vertices).
constexpr int64_t kStaticMaxVertices = 4194304;  // 2^22

// Layout of the scratch array (8-byte words):
//   [0, kStaticMaxVertices)              W(X), cluster weight of label X
//   [kStaticMaxVertices, +kUsedWords)    one byte per label: label in use
//   then kAccWords accumulators (see Acc)
constexpr int64_t kUsedWords = kStaticMaxVertices / 8;
constexpr int kAccWords = 16;
constexpr int64_t kScratchWords = kStaticMaxVertices + kUsedWords + kAccWords;

__device__ __align__(256) unsigned long long g_lc_static_scratch[kScratchWords];

struct Acc {
  unsigned long long phi;       // sum over v of Lambda*w'(v, C[v])
  unsigned long long T;         // sum of edge weights
  unsigned long long V;         // sum of vertex weights
  unsigned long long sw2;       // sum of w(v)^2
  unsigned long long clusters;  // labels in use
  unsigned long long bad_label; // labels outside [0, n)
  unsigned long long bad_col;   // rows outside [0, nnz] and columns outside [0, n) (not followed)
};

struct View {
  long long *W;
  unsigned char *used;
  Acc *acc;
};

__host__ __device__ inline View view_of(void *base) {
  unsigned long long *p = static_cast<unsigned long long *>(base);
  View v;
  v.W = reinterpret_cast<long long *>(p);
  v.used = reinterpret_cast<unsigned char *>(p + kStaticMaxVertices);
  v.acc = reinterpret_cast<Acc *>(p + kStaticMaxVertices + kUsedWords);
  return v;
}

__global__ void k_static_clear(void *base, int64_t n) {
  View s = view_of(base);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    s.W[i] = 0;
    s.used[i] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x < sizeof(Acc) / 8)
    reinterpret_cast<unsigned long long *>(s.acc)[threadIdx.x] = 0;
}

__global__ void k_static_weights(void *base, const int32_t *__restrict__ C,
                                 const int64_t *__restrict__ vw, int64_t n) {
  View s = view_of(base);
  unsigned long long V = 0, sw2 = 0, bad = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = C[v];
    const long long w = vw[v];
    V += (unsigned long long)w;
    sw2 += (unsigned long long)(w * w);
    if (x < 0 || x >= n) {
      bad++;
      continue;
    }
    atomicAdd(reinterpret_cast<unsigned long long *>(&s.W[x]), (unsigned long long)w);
    s.used[x] = 1;
  }
  for (int o = 16; o > 0; o >>= 1) {
    V += __shfl_xor_sync(0xFFFFFFFFu, V, o);
    sw2 += __shfl_xor_sync(0xFFFFFFFFu, sw2, o);
    bad += __shfl_xor_sync(0xFFFFFFFFu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&s.acc->V, V);
    atomicAdd(&s.acc->sw2, sw2);
    if (bad) atomicAdd(&s.acc->bad_label, bad);
  }
}

// One warp per vertex: S(v, C[v]) over the row, then Lambda*w'(v, C[v]).
__global__ void k_static_sweep(void *base, int64_t n, int64_t nnz, const int64_t *__restrict__ rp,
                               const int32_t *__restrict__ col, const int32_t *__restrict__ ew,
                               const int64_t *__restrict__ vw, const int32_t *__restrict__ C,
                               long long mu, long long Lam) {
  View s = view_of(base);
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long phi = 0, T = 0, used = 0, bad = 0;
  for (int64_t v = warp; v < n; v += nw) {
    const int32_t x = C[v];
    const bool ok = x >= 0 && x < n;
    long long self = 0, t = 0;
    int64_t rb = rp[v], re = rp[v + 1];
    if (rb < 0 || rb > re || re > nnz) {  // a malformed row: counted, never read
      if (lane == 0) bad++;
      rb = re = 0;
    }
    for (int64_t e = rb + lane; e < re; e += 32) {
      const int32_t u = col[e];
      t += ew[e];
      if (u < 0 || u >= n) {  // a malformed CSR: counted, never dereferenced
        bad++;
        continue;
      }
      if (ok && C[u] == x) self += ew[e];
    }
    for (int o = 16; o > 0; o >>= 1) {
      self += __shfl_xor_sync(0xFFFFFFFFu, self, o);
      t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
    }
    if (lane == 0) {
      T += (unsigned long long)t;
      if (ok) {
        const long long wv = vw[v];
        phi += (unsigned long long)(Lam * self - mu * wv * (s.W[x] - wv));
      }
      used += s.used[v];
    }
  }
  if (lane == 0) {
    atomicAdd(&s.acc->phi, phi);
    atomicAdd(&s.acc->T, T);
    if (used) atomicAdd(&s.acc->clusters, used);
  }
  if (bad) atomicAdd(&s.acc->bad_col, bad);
}

std::mutex g_mu;
void *g_base[64];
bool g_ready[64];

// The scratch array's device address on the current device (set up once per
// device, with that device current).
int static_base(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ready[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_lc_static_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return LC_ERR_CUDA;
    }
    g_base[dev] = p;
    g_ready[dev] = true;
  }
  *out = g_base[dev];
  return LC_OK;
}

unsigned blocks_for(int64_t items, int per_block) {
  int64_t b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)b;
}

}  // namespace

extern "C" {

LC_API int64_t lc_objective_static_max_vertices(void) { return kStaticMaxVertices; }

LC_API int lc_objective_static(const lc_csr *g, const int64_t *vertex_w, const int32_t *edge_w,
                        int64_t lambda_num, int64_t lambda_den, const int32_t *labels,
                        const lc_opts *opts, lc_result *res) {
  if (!res) return LC_ERR_ARG;
  memset(res, 0, sizeof(*res));
  if (!g || g->n < 0 || g->nnz < 0 || lambda_den <= 0 || lambda_num < 0 || lambda_num > lambda_den)
    return LC_ERR_ARG;
  if (g->n > kStaticMaxVertices) {
    res->error_detail = kStaticMaxVertices;  // the limit that was exceeded
    return LC_ERR_ARG;
  }
  res->lambda_den = lambda_den;
  if (g->n == 0) return LC_OK;
  if (!g->row_ptr || !vertex_w || !labels || (g->nnz > 0 && (!g->col || !edge_w))) return LC_ERR_ARG;
  cudaStream_t s = opts ? (cudaStream_t)opts->stream : nullptr;
  void *base = nullptr;
  int rc = static_base(&base);
  if (rc != LC_OK) return rc;
  const int64_t n = g->n;
  cudaGetLastError();  // an earlier, unrelated launch error is not this call's
  // the row structure bounds every read of the sweep: row_ptr[0] = 0 and
  // row_ptr[n] = nnz (two 8-byte reads into the host stack, no allocation)
  int64_t ends[2] = {-1, -1};
  if (cudaMemcpyAsync(&ends[0], g->row_ptr, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&ends[1], g->row_ptr + n, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return LC_ERR_CUDA;
  }
  if (ends[0] != 0 || ends[1] != g->nnz) return LC_ERR_ARG;
  k_static_clear<<<blocks_for(n, 256), 256, 0, s>>>(base, n);
  k_static_weights<<<blocks_for(n, 256), 256, 0, s>>>(base, labels, vertex_w, n);
  k_static_sweep<<<blocks_for(n * 32, 256), 256, 0, s>>>(base, n, g->nnz, g->row_ptr, g->col, edge_w, vertex_w,
                                                          labels, lambda_num, lambda_den);
  Acc acc;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&acc, view_of(base).acc, sizeof(acc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return LC_ERR_CUDA;
  if (acc.bad_label || acc.bad_col) return LC_ERR_ARG;
  // the sums are exact under the library's guards; beyond them, refuse
  const __int128 T = (long long)acc.T, V = (long long)acc.V;
  if (T < 0 || T >= ((__int128)1 << 31) || V < 0 || V >= ((__int128)1 << 62) ||
      (__int128)lambda_den * T + (__int128)lambda_num * V * V >= ((__int128)1 << 60))
    return LC_ERR_OVERFLOW;
  const long long phi = (long long)acc.phi;
  res->phi = phi;
  res->n_clusters = (int64_t)acc.clusters;
  res->levels = 1;
  res->objective = (double)phi / (double)lambda_den;
  const long long num = phi - (lambda_num ? lambda_num * (long long)acc.sw2 : 0);
  res->modularity = acc.T > 0 ? (double)num / ((double)lambda_den * (double)(long long)acc.T) : 0.0;
  return LC_OK;
}

}  // extern "C"
