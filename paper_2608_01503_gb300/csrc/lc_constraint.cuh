// lc_constraint.cuh — launch interface of lc_constraint.cu (constrained
// coarsening, Section V-B's iteration scheme).
#pragma once

#include "lc_internal.cuh"

namespace lc {

// cnt[v] = number of neighbours u of v with B[u] == B[v] (int32[n]).
void launch_filter_count(const LevelGraph &g, const int32_t *B, int32_t *cnt, cudaStream_t s);
// Writes those edges, in row order, into (col_f, ew_f) at rows rp_f.
void launch_filter_copy(const LevelGraph &g, const int32_t *B, const int64_t *rp_f, int32_t *col_f,
                        int32_t *ew_f, cudaStream_t s);
// B_c[Cd[v]] = B[v] for every v with Cd[v] >= 0 (the members of a coarse
// vertex share their label, so the writes agree).
void launch_coarse_constraint(const int32_t *Cd, const int32_t *B, int32_t *B_c, int64_t n,
                              cudaStream_t s);

}  // namespace lc
