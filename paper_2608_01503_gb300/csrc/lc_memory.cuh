// lc_memory.cuh — where liblc's device scratch comes from.
//
// Every device buffer a call allocates goes through one provider, chosen by
// the call's options: the caller's lc_opts.alloc / lc_opts.dealloc pair
// (e.g. PyTorch's caching allocator, passed by the Python binding), or else
// a stream-ordered memory pool that belongs to the library alone.  The
// private pool keeps freed blocks cached for later calls, so repeated calls
// do not map and unmap memory, but it never changes the device's default
// pool, which other code in the process may use; lc_release_memory() hands
// its cached blocks back to the device.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/lc.h"

namespace lc {

// The library's pool on the current device, created on first use.
cudaMemPool_t private_pool();

// `bytes` of device memory from the call's provider, usable in the order of
// stream s.  LC_ERR_OOM when the provider has none (the callback returned
// NULL or the pool could not grow), LC_ERR_CUDA for other failures.
int dev_alloc(const lc_opts &o, cudaStream_t s, size_t bytes, void **out);
void dev_free(const lc_opts &o, cudaStream_t s, void *p, size_t bytes);

// Device allocations of one call, released together, in stream order, when
// the arena goes out of scope.  `limit` is lc_opts.scratch_limit (0: none);
// `held` and `peak` count the bytes requested.
struct Arena {
  cudaStream_t s;
  lc_opts o;
  std::vector<void *> ptrs;
  std::vector<size_t> sizes;
  int64_t limit = 0, held = 0, peak = 0;
  Arena(cudaStream_t st, const lc_opts &opts) : s(st), o(opts) {}
  Arena(const Arena &) = delete;
  ~Arena() {
    for (size_t i = 0; i < ptrs.size(); ++i)
      if (ptrs[i]) dev_free(o, s, ptrs[i], sizes[i]);
  }
  template <class T>
  int get(T **out, int64_t count) {
    void *p = nullptr;
    const size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
    *out = nullptr;
    if (limit > 0 && held + (int64_t)bytes > limit) return LC_ERR_OOM;
    const int rc = dev_alloc(o, s, bytes, &p);
    if (rc != LC_OK) return rc;
    ptrs.push_back(p);
    sizes.push_back(bytes);
    held += (int64_t)bytes;
    if (held > peak) peak = held;
    *out = (T *)p;
    return LC_OK;
  }
  void release(void *p) {
    for (size_t i = 0; i < ptrs.size(); ++i)
      if (ptrs[i] == p) {
        dev_free(o, s, p, sizes[i]);
        ptrs[i] = nullptr;
        held -= (int64_t)sizes[i];
      }
  }
};

// Upper estimate of the device bytes one lc_cluster_batch call of `count`
// graphs with n vertices and nnz stored edges in total allocates: the
// level-0 scratch exactly (the same sizes the driver requests), plus coarse
// levels whose vertex and edge counts sum to at most those of G_0.  A run
// whose levels shrink more slowly can need more.
int64_t cluster_footprint(int64_t n, int64_t nnz, int count, const lc_opts &o);

}  // namespace lc
