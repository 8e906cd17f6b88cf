"""Pins of the oracle's pLeiden / pLeiden+ (Section V, Algorithms 5 and 6).

* The generator of pLeidenR's random choices is SplitMix64's output
  function; its first outputs from state 0 are the published ones.
* LocalMoveAlt (Section V-A) is re-derived by brute force: the ideal moves
  from Phi differences, each prefix's exact objective change from the pair
  definition of Eq. 1, the committed prefix the best one.
* pLeidenR refines its constraint, keeps vertices that are not well
  connected to their constraint cluster alone, and every refined cluster can
  be produced by Leiden's sequential refinement (Lemma 1): an order exists
  in which each vertex joins an adjacent cluster with w'(v, C) >= 0 while
  w'(C, B minus C) >= 0.
* pLeiden keeps Leiden's per-iteration guarantees (the theorem of Section
  V): every cluster induces a connected subgraph (gamma-connectivity) and no
  two clusters gain by merging (gamma-separation), checked exhaustively.
* Special cases: disjoint cliques, lambda = 0 (connected components)."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as cg

import graphgen as gg
import oracle
from tests import brute


def small_graph(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 36))
    p = float(rng.uniform(0.06, 0.4))
    rp, col, ew = gg.random_graph(n, p, seed, wmax=int(rng.integers(1, 5)))
    kind = seed % 3
    if kind == 0:
        return gg.modularity_inputs(rp, col, ew)
    if kind == 1:
        return gg.cpm_inputs(rp, col, ew, 1, int(rng.integers(2, 20)))
    vw = rng.integers(1, 5, size=n).astype(np.int64)
    return gg.Graph(rp, col, ew, vw, 1, int(rng.integers(3, 30)))


def test_generator_matches_published_splitmix64():
    # SplitMix64 seeded with 0: its first three outputs
    assert oracle.rand(0, 0, 0, 0) == 0xE220A8397B1DCDAF
    assert oracle.rand(0, 0, 0, 1) == 0x6E789E6AA1B965F4
    assert oracle.rand(0, 0, 0, 2) == 0x06C45D188009454F


# ------------------------------------------------------------ LocalMoveAlt

@pytest.mark.parametrize("seed", range(16))
def test_local_move_alt_by_brute_force(seed):
    g = small_graph(seed)
    n = g.n
    A = brute.dense(g.row_ptr, g.col, g.ew)
    P = brute.pair_matrix(A, g.vw, g.lam_num, g.lam_den)
    C = gg.random_labels(n, max(2, n // 3), seed + 1)
    base = brute.pair_objective(P, C)
    # ideal destinations (adjacent clusters, ties to the smallest id, empty rule)
    moves = []
    for v in range(n):
        adjacent = sorted(set(int(C[u]) for u in np.nonzero(A[v])[0]) - {int(C[v])})
        d = {X: brute.pair_objective(P, brute.move(C, v, X)) - base for X in adjacent}
        d_empty = brute.pair_objective(P, brute.move(C, v, oracle.EMPTY)) - base
        best = None
        for X in adjacent:
            if best is None or d[X] > d[best]:
                best = X
        gain = None if best is None else d[best]
        if -d_empty < 0 and (best is None or gain - d_empty < 0):  # gC < 0 and gD < 0
            best, gain = oracle.EMPTY, d_empty
        if best is not None and gain > 0:
            moves.append((v, best))
    got, k = oracle.local_move_alt(g, C)
    if not moves:
        assert k == 0 and np.array_equal(got, C)
        return
    # apply the moves one by one; a move to the empty cluster takes the
    # smallest id unused at that moment (a vertex already alone keeps its id)
    cur = C.astype(np.int64).copy()
    totals, states = [], []
    for v, D in moves:
        if D == oracle.EMPTY:
            if np.sum(cur == cur[v]) == 1:
                D = int(cur[v])
            else:
                D = int(min(set(range(n)) - set(cur.tolist())))
        cur = cur.copy()
        cur[v] = D
        totals.append(brute.pair_objective(P, cur) - base)
        states.append(cur)
    best_k = int(np.argmax(totals))  # first maximum = shortest prefix
    assert totals[best_k] > 0
    assert k == best_k + 1
    assert np.array_equal(got, states[best_k])


# ---------------------------------------------------------------- pLeidenR

def _leidenr_reachable(X, B, A, vw, mu, Lam):
    """Some order of X in which every vertex after the first joins an
    adjacent cluster C with w'(v, C) >= 0 while w'(C, B minus C) >= 0."""
    S = [u for u in range(len(B)) if B[u] == B[X[0]]]
    WB = sum(int(vw[u]) for u in S)
    for perm in itertools.permutations(X):
        ok = True
        for j in range(1, len(perm)):
            C, v = perm[:j], perm[j]
            wvc = sum(int(A[v, u]) for u in C)
            if wvc == 0:
                ok = False
                break
            Wc = sum(int(vw[u]) for u in C)
            ext = sum(int(A[u, x]) for u in C for x in S if x not in C)
            if Lam * wvc - mu * int(vw[v]) * Wc < 0 or Lam * ext - mu * Wc * (WB - Wc) < 0:
                ok = False
                break
        if ok:
            return True
    return False


@pytest.mark.parametrize("seed", range(24))
def test_refinement_properties(seed):
    g = small_graph(seed)
    n = g.n
    A = brute.dense(g.row_ptr, g.col, g.ew)
    B, _, _ = oracle.louvain_plus(g)
    if seed % 4 == 3:
        B = gg.random_labels(n, 2, seed)
    R = oracle.pleiden_refine(g, B, level=seed % 3)
    mu, Lam = g.lam_num, g.lam_den
    for X in np.unique(R):
        mem = [int(v) for v in np.nonzero(R == X)[0]]
        assert len(set(int(B[v]) for v in mem)) == 1  # refines B
        if len(mem) == 1:
            continue
        for v in mem:  # members are well connected to their constraint cluster
            S = [u for u in range(n) if B[u] == B[v] and u != v]
            s_in = sum(int(A[v, u]) for u in S)
            WB = sum(int(g.vw[u]) for u in S)
            assert Lam * s_in - mu * int(g.vw[v]) * WB >= 0
        sub = sp.csr_matrix(A[np.ix_(mem, mem)])
        assert cg.connected_components(sub, directed=False)[0] == 1
        if len(mem) <= 7:
            assert _leidenr_reachable(mem, B, A, g.vw, mu, Lam), (seed, mem)


def test_refinement_with_singleton_constraint_is_singletons():
    g = gg.sbm_planted(n=300, blocks=6, p_in=0.2, p_out=0.01, seed=3)
    R = oracle.pleiden_refine(g, np.arange(g.n, dtype=np.int32))
    assert np.array_equal(R, np.arange(g.n))


# ----------------------------------------------------------------- pLeiden

@pytest.mark.parametrize("seed", range(30))
def test_pleiden_connected_and_separated(seed):
    """Leiden's guarantees after an iteration: connected clusters and no
    pair of clusters whose merge increases the objective."""
    g = small_graph(seed)
    lab, res, _ = oracle.pleiden(g, oracle.Params(uncoarsen=False))
    A = brute.dense(g.row_ptr, g.col, g.ew)
    for X in np.unique(lab):
        idx = np.nonzero(lab == X)[0]
        sub = sp.csr_matrix(A[np.ix_(idx, idx)])
        assert cg.connected_components(sub, directed=False)[0] == 1
    P = brute.pair_matrix(A, g.vw, g.lam_num, g.lam_den)
    base = brute.pair_objective(P, lab)
    assert base == res["phi"]
    cl = np.unique(lab)
    for i in range(len(cl)):
        for j in range(i + 1, len(cl)):
            m = lab.copy()
            m[m == cl[j]] = cl[i]
            assert brute.pair_objective(P, m) <= base


def test_pleiden_bounded_by_exhaustive_optimum():
    for seed in range(6):
        rp, col, ew = gg.random_graph(8, 0.45, seed, wmax=3)
        g = gg.cpm_inputs(rp, col, ew, 1, 4)
        P = brute.pair_matrix(brute.dense(rp, col, ew), g.vw, 1, 4)
        for unc in (False, True):
            _, res, _ = oracle.pleiden(g, oracle.Params(uncoarsen=unc))
            assert res["phi"] <= brute.best_partition_objective(P)


def test_pleiden_disjoint_cliques_and_lambda_zero():
    src, dst = [], []
    for c, size in enumerate((6, 9, 5)):
        base = sum((6, 9, 5)[:c])
        for i in range(size):
            for j in range(i + 1, size):
                src.append(base + i)
                dst.append(base + j)
    rp, col, ew = gg.from_edges(20, np.array(src), np.array(dst))
    g = gg.modularity_inputs(rp, col, ew)
    for unc in (False, True):
        lab, _, _ = oracle.pleiden(g, oracle.Params(uncoarsen=unc))
        parts = {frozenset(np.nonzero(lab == x)[0].tolist()) for x in np.unique(lab)}
        assert parts == {frozenset(range(0, 6)), frozenset(range(6, 15)), frozenset(range(15, 20))}
    rp, col, ew = gg.random_graph(40, 0.04, 7)
    g = gg.cpm_inputs(rp, col, ew, 0, 1)
    lab, _, _ = oracle.pleiden(g, oracle.Params(uncoarsen=False))
    k, comp = cg.connected_components(sp.csr_matrix(brute.dense(rp, col, ew)), directed=False)
    assert len(np.unique(lab)) == k
    for c in range(k):
        assert len(np.unique(lab[comp == c])) == 1


def test_pleiden_initial_clustering_and_plus_not_worse_on_sbm():
    g = gg.sbm_planted(n=1500, blocks=15, p_in=0.06, p_out=0.003, seed=4)
    lab0, r0, _ = oracle.pleiden(g, oracle.Params(uncoarsen=False))
    # feeding pLeiden its own output (an iteration) never lowers the objective
    lab1, r1, _ = oracle.pleiden(g, oracle.Params(uncoarsen=False), C_in=lab0)
    assert r1["phi"] >= r0["phi"]
    with pytest.raises(Exception):
        oracle.pleiden(g, C_in=np.full(g.n, g.n, dtype=np.int32))
