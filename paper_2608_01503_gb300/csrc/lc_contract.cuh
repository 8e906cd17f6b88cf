// lc_contract.cuh — launch interface of lc_contract.cu.
#pragma once

#include "lc_internal.cuh"

namespace lc {

// used[x] = 1 for every label x that some C[v] holds (used: int32[n]).
void launch_mark_used(const int32_t *C, int64_t n, int32_t *used, cudaStream_t s);
// Numbers the used labels (of graphs with keep[g], keep nullable) in
// ascending order: newid[x], gstart[g] = number of such labels before graph
// g's first vertex, gid_next[newid] = graph (nullable).  The total is left in
// *compact_total(scan_tmp, n) on the device.
void launch_number_labels(const int32_t *used, int64_t n, const int32_t *gid, const GraphParam *gp,
                          const uint8_t *keep, int32_t *newid, int32_t *gstart, int32_t *gid_next,
                          int32_t *scan_tmp, cudaStream_t s);
// out[v] = newid[C[v]] (minus gstart[g] if local); -1 where keep[g] == 0.
void launch_relabel(const int32_t *C, const int32_t *newid, int32_t *out, int64_t n, const int32_t *gid,
                    const int32_t *gstart, const uint8_t *keep, int local, cudaStream_t s);
const int32_t *compact_total(const int32_t *scan_tmp, int64_t n);

// Algorithm 4, lines 1-4: bound, offsets (int64[n_c+1]) and coarse vertex weights.
void launch_contract_offsets(const LevelGraph &g, const int32_t *Cd, int64_t n_c, int64_t *bound,
                             int64_t *off, int64_t *vw_c, int64_t *scan_tmp64, cudaStream_t s);
// Algorithm 4, lines 5-12: inserts with unique counting (cnt int32[n_c]).
// Returns the number of kernels launched.
int launch_contract_insert(const LevelGraph &g, const int32_t *Cd, const int64_t *off,
                           unsigned long long *tab, int32_t *cnt, int64_t n_c, int *error,
                           const int32_t *const *lists, const int64_t *counts, const Hubs &hub,
                           cudaStream_t s);
// Coarse row offsets from the unique counts; rp_c[n_c] = nnz_c.
void launch_contract_rowptr(const int32_t *cnt, int64_t n_c, int64_t *rp_c, int64_t *scan_tmp64,
                            cudaStream_t s);
// Algorithm 4, line 13: stream compaction of all table slots into the coarse CSR.
void launch_contract_compact(unsigned long long *tab, int64_t slots, int32_t *col_c, int32_t *ew_c,
                             int32_t *scan_tmp, cudaStream_t s);
// gid[v] for a packed batch with vertex ranges gptr[0..G] (device).
void launch_graph_ids(const int64_t *gptr, int G, int32_t *gid, int64_t n, cudaStream_t s);
// C[v] = vbase_fine(g) + Cnext[Cd[v]] - vbase_coarse(g) (Cd[v] < 0: C[v] = v)
void launch_project(const int32_t *Cd, const int32_t *Cnext, int32_t *C, int64_t n, const int32_t *gid,
                    const GraphParam *gp_fine, const GraphParam *gp_coarse, cudaStream_t s);

}  // namespace lc
