// lc_debug.cu — the registry of the checked build's per-unit fault records,
// and lc_debug_enabled / lc_debug_selftest (lc_debug.cuh says what is
// checked).  In the release build the registry stays empty.
#include <mutex>
#include <vector>

#include "../../include/lc.h"
#include "lc_debug.cuh"

namespace lc {

namespace {
std::mutex &reg_mu() {
  static std::mutex m;
  return m;
}
std::vector<DbgReader> &readers() {
  static std::vector<DbgReader> r;  // filled while the library loads
  return r;
}
}  // namespace

void dbg_register(DbgReader f) {
  std::lock_guard<std::mutex> lk(reg_mu());
  readers().push_back(f);
}

long long dbg_collect(cudaStream_t s, DbgRecord *first) {
  std::lock_guard<std::mutex> lk(reg_mu());
  long long total = 0;
  for (DbgReader f : readers()) {
    DbgRecord r{};
    if (f(s, &r) != 0) continue;  // a unit whose module never loaded
    if (r.count && total == 0 && first) *first = r;
    total += r.count;
  }
  return total;
}

#if LC_DEBUG
// One thread fails one check on purpose; no memory is addressed with the
// failed index.
__global__ void k_dbg_selftest(long long i, long long n) {
  volatile long long sink = LC_IDX(i, n, kDbgSelfTest);
  (void)sink;
}
#endif

}  // namespace lc

extern "C" LC_API int lc_debug_enabled(void) { return LC_DEBUG; }

extern "C" LC_API int lc_debug_selftest(void *stream, int64_t *detail) {
#if LC_DEBUG
  const cudaStream_t s = (cudaStream_t)stream;
  lc::DbgRecord first{};
  lc::dbg_collect(s, nullptr);  // start from clear records
  lc::k_dbg_selftest<<<1, 1, 0, s>>>(7, 3);
  if (cudaGetLastError() != cudaSuccess) return LC_ERR_CUDA;
  const long long n = lc::dbg_collect(s, &first);
  if (detail) *detail = ((int64_t)first.site << 56) | (first.index & ((1ll << 56) - 1));
  return n == 1 && first.site == lc::kDbgSelfTest && first.index == 7 && first.bound == 3 ? LC_OK
                                                                                            : LC_ERR_DEVICE;
#else
  (void)stream;
  if (detail) *detail = 0;
  return LC_ERR_ARG;  // not the checked build
#endif
}
