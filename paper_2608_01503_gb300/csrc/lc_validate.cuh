// lc_validate.cuh — launch interface of lc_validate.cu.
#pragma once

#include "lc_internal.cuh"

namespace lc {

struct GraphStats {
  long long T;    // sum of stored edge weights (2 m_w)
  long long V;    // sum of vertex weights
  long long sw2;  // sum of w(v)^2 (exact when the guards hold)
  unsigned long long fp1, fp2;  // symmetric-edge fingerprints, 0 when symmetric
  unsigned long long err_key;   // (code << 40 | vertex), min over violations; ~0 if none
};

// Sums T, V, sum w^2; with validate: row structure, ranges, loops, weights,
// strictly increasing rows and the symmetry fingerprints.  *st must be
// zeroed with err_key = ~0 beforehand.
// With a packed batch (gid non-null) also per-graph sums Tg, Vg, sw2g
// (zeroed beforehand) and a check that no edge crosses graphs.
void launch_stats(const LevelGraph &g, int validate, GraphStats *st, const int32_t *gid, long long *Tg,
                  long long *Vg, long long *sw2g, cudaStream_t s);
// Reports LC_ERR_ARG for any label outside [0, limit).
void launch_labels_in_range(const int32_t *C, int64_t n, int64_t limit, GraphStats *st,
                            cudaStream_t s);

}  // namespace lc
