// lc_constraint.cu — constrained coarsening (Section V-B, the iteration
// scheme for Louvain+).
//
// A constraint clustering B restricts every coarsening-phase move of v to
// clusters whose members all share B[v].  Every cluster formed under that
// rule lies inside one class of B, so for such clusterings
//   * S(v, X) for an allowed X only involves edges (v,u) with B[u] = B[v],
//   * the afterburner terms of a neighbour u in another class vanish (its
//     C[u] and D[u] lie in its own class, never equal to C[v] or D[v]),
//   * Phi only counts edges inside clusters, hence inside classes.
// The constrained passes on G_l are therefore exactly the unconstrained
// passes on G_l with the edges between classes removed.  The driver runs
// the coarsening passes on that filtered graph (built here), contracts the
// full G_l, and carries B to the coarse level; uncoarsening uses G_l.
#include "lc_constraint.cuh"

namespace lc {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__global__ void __launch_bounds__(kThreads) k_filter_count(LevelGraph g, const int32_t *__restrict__ B,
                                                           int32_t *__restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  for (int64_t v = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); v < g.n;
       v += (int64_t)gridDim.x * kWarps) {
    const int64_t beg = g.rp[v], end = g.rp[v + 1];
    const int32_t Bv = B[v];
    int32_t c = 0;
    for (int64_t e = beg + lane; e < end; e += 32) c += B[__ldg(g.col + e)] == Bv;
    c = __reduce_add_sync(0xFFFFFFFFu, (unsigned)c);
    if (lane == 0) cnt[v] = c;
  }
}

__global__ void __launch_bounds__(kThreads) k_filter_copy(LevelGraph g, const int32_t *__restrict__ B,
                                                          const int64_t *__restrict__ rp_f,
                                                          int32_t *__restrict__ col_f,
                                                          int32_t *__restrict__ ew_f) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  for (int64_t v = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); v < g.n;
       v += (int64_t)gridDim.x * kWarps) {
    const int64_t beg = g.rp[v], end = g.rp[v + 1];
    const int32_t Bv = B[v];
    int64_t pos = rp_f[v];
    for (int64_t base = beg; base < end; base += 32) {
      const int64_t e = base + lane;
      int32_t u = -1;
      bool keep = false;
      if (e < end) {
        u = __ldg(g.col + e);
        keep = B[u] == Bv;
      }
      const unsigned m = __ballot_sync(0xFFFFFFFFu, keep);
      if (keep) {
        const int64_t at = pos + __popc(m & below);
        col_f[at] = u;
        ew_f[at] = __ldg(g.ew + e);
      }
      pos += __popc(m);
    }
  }
}

__global__ void k_coarse_constraint(const int32_t *__restrict__ Cd, const int32_t *__restrict__ B,
                                    int32_t *__restrict__ B_c, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = Cd[v];
    if (x >= 0) B_c[x] = B[v];
  }
}

unsigned warp_grid(int64_t n) {
  const int64_t b = (n + kWarps - 1) / kWarps;
  return (unsigned)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

}  // namespace

void launch_filter_count(const LevelGraph &g, const int32_t *B, int32_t *cnt, cudaStream_t s) {
  if (g.n == 0) return;
  k_filter_count<<<warp_grid(g.n), kThreads, 0, s>>>(g, B, cnt);
}

void launch_filter_copy(const LevelGraph &g, const int32_t *B, const int64_t *rp_f, int32_t *col_f,
                        int32_t *ew_f, cudaStream_t s) {
  if (g.n == 0 || g.nnz == 0) return;
  k_filter_copy<<<warp_grid(g.n), kThreads, 0, s>>>(g, B, rp_f, col_f, ew_f);
}

void launch_coarse_constraint(const int32_t *Cd, const int32_t *B, int32_t *B_c, int64_t n,
                              cudaStream_t s) {
  if (n == 0) return;
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  k_coarse_constraint<<<(unsigned)b, 256, 0, s>>>(Cd, B, B_c, n);
}

}  // namespace lc
