"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check compares the oracle with something other than itself: the pair
definition of Eq. 1 evaluated densely, exhaustive search over partitions,
the networkx modularity routine, scipy's connected components, a membership
matrix product for the coarse graph, and hand-derived closed forms stored in
tests/golden/.  A dropped term, a wrong sign or index, or a transposed
operand in the oracle fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny(n, p, seed, wmax=3, vw_mode="rand", lam=(1, 7)):
    rp, col, ew = gg.random_graph(n, p, seed, wmax=wmax)
    rng = np.random.default_rng(seed + 99)
    if vw_mode == "rand":
        vw = rng.integers(1, 5, size=n).astype(np.int64)
    elif vw_mode == "deg":
        vw = gg.weighted_degree(rp, ew)
        vw = np.maximum(vw, 1)
    else:
        vw = np.ones(n, np.int64)
    return gg.Graph(rp, col, ew, vw, lam[0], lam[1], f"tiny{n}_{seed}")


CASES = [(n, p, s, lam) for s, (n, p, lam) in enumerate(
    [(6, 0.5, (1, 7)), (8, 0.4, (1, 9)), (9, 0.35, (2, 11)), (7, 0.6, (0, 1)), (8, 0.3, (1, 1)),
     (10, 0.3, (1, 13)), (5, 0.8, (3, 10)), (9, 0.5, (1, 30))])]


# ------------------------------------------------------------------ Eq. 1 ---

@pytest.mark.parametrize("n,p,seed,lam", CASES)
def test_objective_equals_pair_definition(n, p, seed, lam):
    g = tiny(n, p, seed, lam=lam)
    P = brute.pair_matrix(brute.dense(g.row_ptr, g.col, g.ew), g.vw, g.lam_num, g.lam_den)
    for k in (1, 2, 3, n):
        lab = gg.random_labels(n, k, seed * 7 + k)
        assert oracle.objective(g, lab) == brute.pair_objective(P, lab)


def test_objective_singletons_is_zero():
    g = tiny(9, 0.5, 3)
    assert oracle.objective(g, np.arange(9, dtype=np.int32)) == 0


# -------------------------------------------------------- Section II-A gain ---

@pytest.mark.parametrize("n,p,seed,lam", CASES)
def test_gain_is_half_the_objective_delta(n, p, seed, lam):
    """2 w'(v,C_i) - 2 w'(v,C[v]) is the objective delta of moving v (Section II-A)."""
    g = tiny(n, p, seed, lam=lam)
    P = brute.pair_matrix(brute.dense(g.row_ptr, g.col, g.ew), g.vw, g.lam_num, g.lam_den)
    lab = gg.random_labels(n, 3, seed)
    base = brute.pair_objective(P, lab)
    for v in range(n):
        gc = oracle.gain(g, lab, v, int(lab[v]))
        for X in list(range(n)) + [oracle.EMPTY]:
            if X == lab[v]:
                continue
            if X >= 0 and not np.any(lab == X):
                continue  # not a cluster of C
            after = brute.pair_objective(P, brute.move(lab, v, X))
            assert after - base == 2 * (oracle.gain(g, lab, v, X) - gc)


# --------------------------------------------- Algorithm 2 + 3, pass level ---

def _order_key(v, delta, Lam, eps=(1, 10), seed=0):
    # (earlier first): bigger epsilon bucket, then smaller hash, then smaller id
    q = (eps[1] * int(delta)) // (eps[0] * Lam)
    return (-q, brute.fmix32(v ^ seed), v)


@pytest.mark.parametrize("n,p,seed,lam", CASES)
def test_pass_destinations_candidates_and_afterburner(n, p, seed, lam):
    """Every pass of the oracle, checked by brute force through Phi differences:
    D[v] maximises the objective after moving v (ties -> smallest id) over
    adjacent clusters, the empty-cluster rule and the candidate test of
    Algorithm 2 hold, and each afterburner value equals v's exact gain once its
    earlier adjacent candidates have moved (Algorithm 3)."""
    g = tiny(n, p, seed, lam=lam)
    A = brute.dense(g.row_ptr, g.col, g.ew)
    P = brute.pair_matrix(A, g.vw, g.lam_num, g.lam_den)
    params = oracle.Params()
    for start in (np.arange(n, dtype=np.int32), gg.random_labels(n, 3, seed + 5)):
        _, _, events = oracle.local_move(g, start, params, trace=True)
        assert len(events) == params.pass_limit + 1
        for ev in events:
            if ev["kind"] != "pass":
                continue
            C, D = ev["C_before"], ev["D"]
            phi_n, phi_d = params.phi[ev["pass"] - 1]
            base = brute.pair_objective(P, C)
            gains = {}
            for v in range(n):
                adjacent = sorted(set(int(C[u]) for u in np.nonzero(A[v])[0]) - {int(C[v])})
                # 2 (g(v,X) - g(v,C[v])) by brute force
                d2 = {X: brute.pair_objective(P, brute.move(C, v, X)) - base for X in adjacent}
                d_empty = brute.pair_objective(P, brute.move(C, v, oracle.EMPTY)) - base
                gC2 = -d_empty  # 2 g(v,C[v]) since g(v, empty) = 0
                best = None
                for X in adjacent:
                    if best is None or d2[X] > d2[best]:
                        best = X
                gD2 = None if best is None else d2[best] + gC2
                if gC2 < 0 and (best is None or gD2 < 0):
                    best, gD2 = oracle.EMPTY, 0
                exp_D = oracle.NONE if best is None else best
                assert D[v] == exp_D, (ev["level"], ev["pass"], v)
                in_L = best is not None and phi_d * gD2 >= (phi_d - phi_n) * gC2
                assert bool(ev["in_L"][v]) == in_L
                if best is not None:
                    assert 2 * ev["delta"][v] == gD2 - gC2
                gains[v] = gD2
            # Algorithm 3 semantics
            L = [v for v in range(n) if ev["in_L"][v]]
            keys = {v: _order_key(v, ev["delta"][v], g.lam_den) for v in L}
            for v in L:
                prior = [u for u in L if A[v, u] and keys[u] < keys[v]]
                Cp = np.array(C, dtype=np.int64)
                for u in prior:
                    Cp = brute.move(Cp, u, int(D[u]))
                b0 = brute.pair_objective(P, Cp)
                b1 = brute.pair_objective(P, brute.move(Cp, v, int(D[v])))
                assert 2 * ev["adj"][v] == b1 - b0
                assert bool(ev["in_M"][v]) == (ev["adj"][v] >= 0)
            # Update: movers take D (a fresh singleton for the empty cluster)
            Ca = ev["C"]
            for v in range(n):
                if ev["in_M"][v] and D[v] >= 0:
                    assert Ca[v] == D[v]
                elif ev["in_M"][v]:
                    assert np.sum(Ca == Ca[v]) == 1
                else:
                    assert Ca[v] == C[v]
            assert ev["phi"] == brute.pair_objective(P, Ca)


def test_priority_order_respects_epsilon():
    """Candidates whose deltas differ by at least epsilon are ordered by delta
    (Section IV-A-1)."""
    rng = np.random.default_rng(1)
    Lam = 1000
    deltas = rng.integers(-5000, 5000, size=300)
    for _ in range(2000):
        u, v = rng.integers(0, 300, size=2)
        if u == v:
            continue
        if deltas[u] - deltas[v] >= Lam // 10:
            assert _order_key(u, deltas[u], Lam) < _order_key(v, deltas[v], Lam)


def test_node_optimal_when_no_candidates():
    """A pass with an empty candidate list leaves a node-optimal clustering:
    no single move (adjacent cluster or a new one) raises the objective
    (Section II-B, node optimality)."""
    seen = 0
    for seed in range(12):
        g = tiny(9, 0.4, 100 + seed, lam=(1, 9))
        A = brute.dense(g.row_ptr, g.col, g.ew)
        P = brute.pair_matrix(A, g.vw, g.lam_num, g.lam_den)
        _, _, events = oracle.local_move(g, np.arange(9, dtype=np.int32), trace=True)
        for ev in events:
            if ev["kind"] == "pass" and ev["count_L"] == 0:
                seen += 1
                C = ev["C_before"]
                base = brute.pair_objective(P, C)
                for v in range(9):
                    for X in set(C.tolist()) | {oracle.EMPTY}:
                        if X != C[v]:
                            assert brute.pair_objective(P, brute.move(C, v, X)) <= base
    assert seen > 0


# ---------------------------------------------------------- contraction ---

@pytest.mark.parametrize("n,p,seed,lam", CASES)
def test_contraction_matches_membership_product(n, p, seed, lam):
    g = tiny(n, p, seed, lam=lam)
    A = brute.dense(g.row_ptr, g.col, g.ew)
    for k in (1, 2, 4):
        lab = gg.random_labels(n, k, seed + k)
        _, lab = np.unique(lab, return_inverse=True)
        lab = lab.astype(np.int32)
        n_c = int(lab.max()) + 1
        rp, col, ew, vw = oracle.contract(g, lab, n_c)
        Ac = brute.coarse_dense(A, lab, n_c)
        assert np.array_equal(brute.dense(rp, col, ew), Ac)
        assert np.array_equal(vw, np.bincount(lab, weights=g.vw, minlength=n_c).astype(np.int64))
        for x in range(n_c):  # rows sorted, no self-loops
            row = col[rp[x]:rp[x + 1]]
            assert np.all(np.diff(row) > 0) and not np.any(row == x)
        internal = int(sum(A[u, v] for u in range(n) for v in range(n) if lab[u] == lab[v]))
        assert int(ew.sum()) == int(g.ew.sum()) - internal


@pytest.mark.parametrize("n,p,seed,lam", CASES)
def test_projected_objective_offset_is_constant(n, p, seed, lam):
    """Section III-A: the objective of a coarse clustering differs from that of
    the induced fine clustering by a constant, Phi(C) of the contracting
    clustering."""
    g = tiny(n, p, seed, lam=lam)
    lab = gg.random_labels(n, 3, seed)
    _, lab = np.unique(lab, return_inverse=True)
    lab = lab.astype(np.int32)
    n_c = int(lab.max()) + 1
    rp, col, ew, vw = oracle.contract(g, lab, n_c)
    gc = gg.Graph(rp, col, ew, vw, g.lam_num, g.lam_den)
    off = oracle.objective(g, lab)
    for s in range(4):
        cl = gg.random_labels(n_c, 2, s)
        assert oracle.objective(g, cl[lab]) == oracle.objective(gc, cl) + off


# ----------------------------------------------------- whole Algorithm 1 ---

@pytest.mark.parametrize("seed", range(10))
def test_louvain_plus_bounded_by_exhaustive_optimum(seed):
    """NP-hard objective (Section II-A): the heuristic can only reach the
    exhaustive optimum from below."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 10))
    lam = [(1, 9), (1, 5), (2, 7), (1, 20)][seed % 4]
    g = tiny(n, 0.45, 500 + seed, lam=lam, vw_mode=["rand", "deg", "one"][seed % 3])
    P = brute.pair_matrix(brute.dense(g.row_ptr, g.col, g.ew), g.vw, g.lam_num, g.lam_den)
    labels, res, _ = oracle.louvain_plus(g)
    phi = brute.pair_objective(P, labels)
    assert phi == res["phi"]
    assert res["objective"] == phi / g.lam_den
    opt = brute.best_partition_objective(P)
    assert phi <= opt
    assert phi >= 0  # never worse than the singleton start (best-of)
    assert sorted(set(labels.tolist())) == list(range(res["n_clusters"]))


def test_disjoint_cliques_found_exactly():
    """Disjoint unit cliques under CPM lambda = 1/2: the optimum is the cliques
    (every intra pair gains 1/2, every inter pair loses 1/2)."""
    sizes = [3, 4, 5, 2]
    src, dst, off = [], [], 0
    for s in sizes:
        for a in range(s):
            for b in range(a + 1, s):
                src.append(off + a)
                dst.append(off + b)
        off += s
    rp, col, ew = gg.from_edges(off, src, dst)
    g = gg.cpm_inputs(rp, col, ew, 1, 2)
    labels, res, _ = oracle.louvain_plus(g)
    expect = np.repeat(np.arange(len(sizes)), sizes)
    assert np.array_equal(labels, expect)
    assert res["phi"] == sum(s * (s - 1) for s in sizes)  # Lambda*(1-lambda)*s(s-1)


def test_lambda_zero_reaches_connected_components():
    """lambda = 0 (label propagation, Section II-A): the optimum merges each
    connected component; the method reaches it on these small graphs."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    for seed in range(6):
        rp, col, ew = gg.random_graph(30, 0.06, 900 + seed, wmax=4)
        g = gg.Graph(rp, col, ew, np.ones(30, np.int64), 0, 1)
        labels, res, _ = oracle.louvain_plus(g)
        A = sp.csr_matrix((ew, col, rp), shape=(30, 30))
        k, comp = connected_components(A, directed=False)
        assert res["phi"] <= int(ew.sum())  # Lambda * total ordered weight
        _, canon = np.unique(comp, return_inverse=True)
        # same partition up to renaming
        pairs_a = comp[:, None] == comp[None, :]
        pairs_b = labels[:, None] == labels[None, :]
        assert np.array_equal(pairs_a, pairs_b), seed


def test_modularity_matches_networkx():
    nx = pytest.importorskip("networkx")
    g = gg.sbm_planted(n=600, blocks=6, p_in=0.08, p_out=0.004, seed=3)
    labels, res, _ = oracle.louvain_plus(g)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    r = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    m = r < g.col
    G.add_weighted_edges_from(zip(r[m].tolist(), g.col[m].tolist(), g.ew[m].tolist()))
    comms = [set(np.nonzero(labels == c)[0].tolist()) for c in range(res["n_clusters"])]
    q = nx.community.modularity(G, comms, weight="weight")
    assert abs(q - res["modularity"]) <= 1e-12 * max(1.0, abs(q))


def test_sbm_planted_quality_band():
    """Planted-partition SBM (10,000 vertices, 100 blocks): the method's
    modularity is within 0.01 of the planted partition's (a band, not parity)."""
    g = gg.sbm_planted()
    labels, res, _ = oracle.louvain_plus(g)
    planted = np.repeat(np.arange(100), 100).astype(np.int32)
    phi_p = oracle.objective(g, planted)
    q_p = (phi_p - int((g.vw.astype(object) ** 2).sum())) / (g.lam_den * int(g.ew.sum()))
    assert res["modularity"] >= q_p - 0.01


# --------------------------------------------------------------- golden ---

def _golden_cases():
    with open(os.path.join(GOLDEN, "closed_forms.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_golden_closed_forms(case):
    n = case["n"]
    src = [e[0] for e in case["edges"]]
    dst = [e[1] for e in case["edges"]]
    rp, col, ew = gg.from_edges(n, src, dst)
    if case["objective"] == "modularity":
        g = gg.modularity_inputs(rp, col, ew)
    else:
        g = gg.cpm_inputs(rp, col, ew, *case["lambda"])
    labels = np.array(case["labels"], dtype=np.int32)
    phi = oracle.objective(g, labels)
    num, den = case["phi_over_Lambda"]
    assert phi * den == num * g.lam_den
    if "modularity" in case:
        mnum, mden = case["modularity"]
        sw2 = int((g.vw.astype(object) ** 2).sum())
        assert (phi - g.lam_num * sw2) * mden == mnum * g.lam_den * int(ew.sum())
    if case.get("method_reaches"):
        lab2, res, _ = oracle.louvain_plus(g)
        assert res["phi"] == phi


def test_best_of_keeps_the_earliest_maximum():
    """Algorithm 2 replaces C_out only on a strict lambdaCC improvement, so
    among tied maxima the earliest state (the input first) is returned.
    The seeds below give two different states of equal objective."""
    checked = 0
    for seed in (0, 4, 8, 25, 37):
        rng = np.random.default_rng(seed)
        n = int(rng.integers(4, 9))
        rp, col, ew = gg.random_graph(n, float(rng.uniform(0.3, 0.8)), seed, wmax=int(rng.integers(1, 3)))
        lam = [(1, 2), (1, 3), (1, 4), (2, 5)][seed % 4]
        g = gg.Graph(rp, col, ew, np.ones(n, np.int64), lam[0], lam[1])
        P = brute.pair_matrix(brute.dense(rp, col, ew), g.vw, g.lam_num, g.lam_den)
        start = np.arange(n, dtype=np.int32) if seed % 2 == 0 else gg.random_labels(n, 2, seed)
        C_out, phi_out, events = oracle.local_move(g, start, trace=True)
        states = [start] + [e["C"] for e in events if e["kind"] == "pass"]
        phis = [brute.pair_objective(P, s) for s in states]
        first = int(np.argmax(phis))  # argmax returns the first maximum
        assert np.array_equal(C_out, states[first])
        assert phi_out == phis[first]
        checked += sum(1 for s, f in zip(states, phis) if f == phis[first] and not np.array_equal(s, states[first]))
    assert checked > 0
