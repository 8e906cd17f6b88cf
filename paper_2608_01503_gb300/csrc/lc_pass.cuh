// lc_pass.cuh — launch interface of the local-move pass kernels (lc_pass.cu).
#pragma once

#include "lc_internal.cuh"

namespace lc {

// Everything one pass kernel reads or writes (device pointers, by value).
struct PassArgs {
  LevelGraph g;
  Method m;
  const int32_t *gid;     // graph of each vertex of a packed batch (nullptr: one graph)
  const GraphParam *gp;   // [G] per-graph lambda, vertex base, active flag
  int32_t G;
  long long *gself;       // batch only: per-vertex g(v, C[v]) for the per-graph objective
  long long *phi_acc;     // [G] objective of the clustering entering the pass
  long long *phi_out;     // [G] objective of C_out
  int *improved;          // [G] last best-of test
  int32_t *C;       // clustering entering the pass (updated by the apply step)
  int64_t *W;       // W(X) for X in [0, n)
  int32_t *D;       // destination of candidates; kNone for non-candidates
  int64_t *delta;   // g(v, D[v]) - g(v, C[v]) of candidates
  AbRec *ab;        // per-pass {C, D, epsilon bucket of delta} (Section IV-A-1 order)
  uint8_t *M;       // afterburner survivors
  Scalars *sc;
  unsigned long long *gtab;  // clean global hash scratch, >= 2 nnz slots
  int32_t phi_n, phi_d;      // temperature of this pass
  const int *phi_live;       // non-null: the temperature is sc->phi_live (graph replays)
  Hubs hub;                  // chunk plan of the hub bin of this level
  // kept tables: each vertex's S(v, .) in its gtab region (tab_cap slots)
  int32_t tab_build;         // this aggregation pass also writes the tables out
  int32_t tab_reset;         // this table pass clears the tables as it reads them
  int32_t *Cprev;            // [n] label before the last apply, of its movers
  int32_t *dirty;            // [n] 1: the table overflowed and is rebuilt (zero between passes)
  int32_t *dirty_list;       // [n] those vertices, sc->tab_dirty of them
  int2 *upd_list;            // chunks {mover, chunk} of the movers' rows, listed by the
                             // apply step when tables are kept (else nullptr)
  int32_t *movers;           // movers that are not hubs, listed by the apply step of a
                             // call's last pass (else nullptr), sc->n_movers
  long long *obj;            // [4 G] per graph: Phi entering the last pass, Q entering it,
                             // Q after it, change of IN by its moves (objective update)
  int64_t hub_min;           // rows longer than this are hubs (BinPlan::hub_min)
  // afterburner: candidate bitmap (bit v of word v / 32) and the candidates
  // of each group, listed by the record pass into ab_list[ab_off[g] ...)
  uint32_t *inL;
  AbWork *ab_list;
  int64_t ab_off[kAbGroups];  // start of group g (the offset of its first bin)
  int64_t ab_max[kAbGroups];  // largest degree in group g (BinPlan)
  int32_t ab_gs[kAbGroups];   // threads per candidate in group g (BinPlan)
};

// Vertex lists of the degree bins of one level (stable: ascending ids).
struct Bins {
  int32_t *lists;    // device, n entries, bin after bin
  int32_t *offs;     // device, kBins + 1 entries
  VRec *recs;        // device, n entries: the vertex records of `lists`, same order
  const int32_t *list[kBins];
  const VRec *rec[kBins];
  int64_t count[kBins];
};

// Bins are stored one after the other, so a run of bins is one list.
struct BinRange {
  const int32_t *list;
  const VRec *rec;
  int64_t count;
};
inline BinRange bin_range(const Bins &b, int lo, int hi) {
  BinRange r{b.list[lo], b.rec[lo], 0};
  for (int k = lo; k <= hi; ++k) r.count += b.count[k];
  return r;
}

void configure_kernels();
// Builds b.lists / b.offs on the stream; the caller copies b.offs to the host
// and fills b.list / b.count (see finish_bins).
void build_bins(const LevelGraph &g, const BinPlan &plan, Bins &b, int32_t *scan_tmp, cudaStream_t s);
void finish_bins(Bins &b, const int32_t *h_offs);
// Fills b.recs from b.lists (gid: graph of each vertex, or null for one graph).
void launch_vertex_records(const LevelGraph &g, const int32_t *gid, Bins &b, cudaStream_t s);

// Launchers return the number of kernels they launched.
void launch_hub_rows(const int64_t *rp, const int32_t *vtx, int H, int64_t *out, cudaStream_t s);
// Resets the pass counters; advance = 1 also loads the pass's temperature
// from the device schedule (sc->phi_tab) and moves to the next pass.
void launch_pass_begin(Scalars *sc, cudaStream_t s, int advance = 0);
int launch_first_pass(const PassArgs &a, const Bins &b, cudaStream_t s);
int launch_move(const PassArgs &a, const Bins &b, cudaStream_t s);
// Fills the afterburner groups' list offsets and degree bounds of a level.
void set_ab_groups(PassArgs &a, const Bins &b, const BinPlan &plan);
int launch_afterburner(const PassArgs &a, const Bins &b, cudaStream_t s);
// Ablations of the afterburner: every candidate moves, or (mlh) all but a
// vertex alone in its cluster whose destination is another one-vertex
// cluster with a larger label.  size: int32[n] scratch.
int launch_symmetry_ablation(const PassArgs &a, bool mlh, int32_t *size, cudaStream_t s);
int launch_objective(const PassArgs &a, const Bins &b, cudaStream_t s);
// The objective of each graph's state after a call's last pass, from the
// state entering it.  launch_last_pass_enter runs at the start of the last
// pass (Q of W before its update), launch_save_phi_enter after its move step
// and per-graph sums (Phi entering), launch_final_objective after its update
// (the movers' edges, Q after; needs the pass's M and Cprev): Phi into
// phi_acc[g].
int launch_last_pass_enter(const PassArgs &a, cudaStream_t s);
int launch_save_phi_enter(const PassArgs &a, cudaStream_t s);
int launch_final_objective(const PassArgs &a, cudaStream_t s);
// Kept tables (Section IV-A-3): applies the last pass's moves to the tables
// of the movers' neighbours (rebuilding any that overflow), then the argmax
// and candidate test of Algorithm 2, read from the tables for vertices of
// degree above kTabMinDeg and aggregated from the CSR for the others.
int launch_table_pass(const PassArgs &a, const Bins &b, cudaStream_t s);
// Entries of PassArgs::upd_list a level of n vertices and nnz stored edges
// may need.
inline int64_t upd_list_size(int64_t n, int64_t nnz) { return n + nnz / kUpdChunk + 1; }
// Scratch of the update step (all [n] of the level).
struct ApplyScratch {
  uint8_t *E;
  int32_t *used, *freelist, *freepos, *mrank, *scan_tmp;
};
// Update step: moves, W, then ids for movers to new empty clusters.
int launch_apply(const PassArgs &a, const ApplyScratch &w, cudaStream_t s);
// Batch only: per-graph sums of the recorded g(v, C[v]) into phi_acc.
int launch_graph_sums(const PassArgs &a, cudaStream_t s);
// Per-graph best-of test and copy of improved graphs' labels into C_out.
int launch_bestof(const PassArgs &a, int32_t *C_out, cudaStream_t s);
// phi_final[g] = phi_out[g] for every graph active in the call (gp[g].active).
int launch_keep_phi(const PassArgs &a, long long *phi_final, cudaStream_t s);
void launch_iota(int32_t *C, int64_t n, cudaStream_t s);
void launch_cluster_weights(const int32_t *C, const int64_t *vw, int64_t *W, int64_t n,
                            cudaStream_t s);

}  // namespace lc
