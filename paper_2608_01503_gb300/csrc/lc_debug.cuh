// lc_debug.cuh — the checked build of liblc (compiled with -DLC_DEBUG=1).
//
// The release kernels trust what they index with once the inputs passed the
// host's checks: a column read from the CSR, a cluster label read from C, a
// destination read from D, a coarse id read from the contraction's map.  The
// checked build tests each of those indexes against the size of the array it
// is about to address.  A failed check does not fault and does not stop the
// kernel: it records the first failure of its translation unit (site, index,
// bound), replaces the index by 0 so that the access stays inside the array,
// and the host turns the record into LC_ERR_DEVICE at the end of the call
// (lc_result.error_detail = site << 56 | index & (2^56 - 1)).  Hash tables
// are bounded in both builds: a probe sequence never runs past its table's
// capacity and an overrun sets Scalars::error; the checked build also
// records where it happened.
//
// In the release build every macro below is the bare index and nothing is
// recorded, so the two builds run the same arithmetic on valid inputs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#ifndef LC_DEBUG
#define LC_DEBUG 0
#endif

namespace lc {

// Where a check failed.
enum DbgSite : int {
  kDbgColumn = 1,     // a neighbour id read from the CSR outside [0, n)
  kDbgLabel = 2,      // a cluster label read from C outside [0, n)
  kDbgDest = 3,       // a destination read from D outside [0, n)
  kDbgProbe = 4,      // a hash probe sequence that reached its table's capacity
  kDbgCoarse = 5,     // a coarse vertex id outside [0, n_c)
  kDbgSelfTest = 15,  // lc_debug_selftest's deliberate failure (no access made)
};

struct DbgRecord {
  unsigned int count;  // failed checks since the last collection
  int site;            // DbgSite of the first one
  long long index, bound;
};

// Host side: every translation unit of the checked build registers a reader
// of its own record (a __device__ variable is per unit without relocatable
// device code).  dbg_collect reads and clears all of them on the stream and
// returns the number of failed checks, the first unit's record in *first.
using DbgReader = int (*)(cudaStream_t, DbgRecord *);
void dbg_register(DbgReader f);
long long dbg_collect(cudaStream_t s, DbgRecord *first);

#if LC_DEBUG

namespace {

__device__ DbgRecord g_dbg_record;

__device__ __noinline__ void dbg_fail(int site, long long i, long long n) {
  if (atomicAdd(&g_dbg_record.count, 1u) == 0u) {
    g_dbg_record.site = site;
    g_dbg_record.index = i;
    g_dbg_record.bound = n;
  }
}

__device__ __forceinline__ long long dbg_index(long long i, long long n, int site) {
  if (i >= 0 && i < n) return i;
  dbg_fail(site, i, n);
  return 0;
}

int dbg_read_unit(cudaStream_t s, DbgRecord *out) {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_dbg_record) != cudaSuccess) return -1;
  if (cudaMemcpyAsync(out, p, sizeof(DbgRecord), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemsetAsync(p, 0, sizeof(DbgRecord), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return -1;
  return 0;
}

struct DbgRegistrar {
  DbgRegistrar() { dbg_register(&dbg_read_unit); }
};
DbgRegistrar g_dbg_registrar;

}  // namespace

template <class T>
__device__ __forceinline__ T dbg_index_t(T i, long long n, int site) {
  return (T)dbg_index((long long)i, n, site);
}

// i (of any integer type) checked against [0, n); 0 in its place on failure.
#define LC_IDX(i, n, site) ::lc::dbg_index_t((i), (long long)(n), (site))
// records a failure found by the caller's own test (no index replaced)
#define LC_DBG_FAIL(site, i, n) ::lc::dbg_fail((site), (long long)(i), (long long)(n))

#else

#define LC_IDX(i, n, site) (i)
#define LC_DBG_FAIL(site, i, n) ((void)0)

#endif

}  // namespace lc
