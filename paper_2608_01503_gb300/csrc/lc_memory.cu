// lc_memory.cu — device memory provider of liblc (see lc_memory.cuh).
#include <mutex>

#include "lc_memory.cuh"

namespace lc {

cudaMemPool_t private_pool() {
  static std::mutex mtx;
  static std::vector<cudaMemPool_t> pools;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(mtx);
  if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    // keep freed blocks for the library's later calls (this pool only)
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
    pools[dev] = p;
  }
  return pools[dev];
}

int dev_alloc(const lc_opts &o, cudaStream_t s, size_t bytes, void **out) {
  *out = nullptr;
  if (o.alloc) {
    void *p = o.alloc(o.alloc_ctx, bytes, (void *)s);
    if (!p) return LC_ERR_OOM;
    *out = p;
    return LC_OK;
  }
  cudaMemPool_t pool = private_pool();
  if (!pool) return LC_ERR_CUDA;
  void *p = nullptr;
  const cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? LC_ERR_OOM : LC_ERR_CUDA;
  }
  *out = p;
  return LC_OK;
}

void dev_free(const lc_opts &o, cudaStream_t s, void *p, size_t bytes) {
  if (!p) return;
  if (o.alloc)
    o.dealloc(o.alloc_ctx, p, bytes, (void *)s);
  else
    cudaFreeAsync(p, s);
}

}  // namespace lc

extern "C" LC_API int lc_release_memory(void) {
  cudaMemPool_t pool = lc::private_pool();
  if (!pool) return LC_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemPoolTrimTo(pool, 0) != cudaSuccess) {
    cudaGetLastError();
    return LC_ERR_CUDA;
  }
  return LC_OK;
}
