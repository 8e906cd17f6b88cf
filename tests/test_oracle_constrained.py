"""Pins of the oracle's constrained and iterated Louvain+ (Section V-B, the
note on iterating Louvain+): during coarsening a vertex may join a cluster
only if every member shares its constraint label; uncoarsening is free.

Checked against brute force on the definition (every coarsening pass of
level 0 re-derived from Phi differences over the allowed clusters), the
invariant that the coarsening output refines the constraint, and the two
special cases that reduce to known results (one constraint class = plain
Louvain+; all-distinct classes = no move at all)."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from tests import brute
from tests.test_oracle_pins import CASES, tiny


@pytest.mark.parametrize("n,p,seed,lam", CASES)
def test_constrained_pass_destinations(n, p, seed, lam):
    g = tiny(n, p, seed, lam=lam)
    A = brute.dense(g.row_ptr, g.col, g.ew)
    P = brute.pair_matrix(A, g.vw, g.lam_num, g.lam_den)
    params = oracle.Params()
    B = gg.random_labels(n, 2, seed + 11)
    _, _, events = oracle.louvain_plus_constrained(g, B, params, trace_passes=True)
    checked = 0
    for ev in events:
        if ev["kind"] != "pass" or ev["level"] != 0 or ev["phase"] != "coarsen":
            continue
        C, D = ev["C_before"], ev["D"]
        phi_n, phi_d = params.phi[ev["pass"] - 1]
        base = brute.pair_objective(P, C)
        for v in range(n):
            members = lambda X: np.nonzero(C == X)[0]
            adjacent = sorted(set(int(C[u]) for u in np.nonzero(A[v])[0]) - {int(C[v])})
            allowed = [X for X in adjacent if all(B[u] == B[v] for u in members(X))]
            d2 = {X: brute.pair_objective(P, brute.move(C, v, X)) - base for X in allowed}
            gC2 = -(brute.pair_objective(P, brute.move(C, v, oracle.EMPTY)) - base)
            best = None
            for X in allowed:
                if best is None or d2[X] > d2[best]:
                    best = X
            gD2 = None if best is None else d2[best] + gC2
            if gC2 < 0 and (best is None or gD2 < 0):
                best, gD2 = oracle.EMPTY, 0
            assert D[v] == (oracle.NONE if best is None else best), (ev["pass"], v)
            in_L = best is not None and phi_d * gD2 >= (phi_d - phi_n) * gC2
            assert bool(ev["in_L"][v]) == in_L
            checked += 1
        # every cluster after the pass still lies inside one constraint class
        Ca = ev["C"]
        for X in np.unique(Ca):
            assert len(set(B[Ca == X].tolist())) == 1
    assert checked > 0


@pytest.mark.parametrize("seed", range(6))
def test_coarsening_output_refines_the_constraint(seed):
    """Without uncoarsening, every output cluster lies inside one constraint
    class, on graphs that coarsen over several levels."""
    g = gg.sbm_planted(n=400, blocks=8, p_in=0.15, p_out=0.01, seed=seed)
    B = gg.random_labels(g.n, 3, seed) if seed % 2 else (np.arange(g.n) * 5 // g.n).astype(np.int32)
    lab, res, _ = oracle.louvain_plus_constrained(g, B, oracle.Params(uncoarsen=False))
    assert res["levels"] >= 2
    for X in np.unique(lab):
        assert len(set(B[lab == X].tolist())) == 1
    # with uncoarsening the result may cross classes, and it is never worse
    # than its own coarsening output projected (best-of keeps the input)
    lab2, res2, _ = oracle.louvain_plus_constrained(g, B)
    assert res2["phi"] >= res["phi"]


@pytest.mark.parametrize("n,p,seed,lam", CASES)
def test_single_class_equals_plain(n, p, seed, lam):
    g = tiny(n, p, seed, lam=lam)
    a, ra, _ = oracle.louvain_plus(g)
    b, rb, _ = oracle.louvain_plus_constrained(g, np.full(n, 7, dtype=np.int32))
    assert np.array_equal(a, b) and ra == rb


def test_distinct_classes_move_nothing():
    g = gg.sbm_planted(n=300, blocks=6, p_in=0.2, p_out=0.01, seed=1)
    lab, res, _ = oracle.louvain_plus_constrained(g, np.arange(g.n, dtype=np.int32))
    assert res["n_clusters"] == g.n and res["phi"] == 0 and res["levels"] == 1


def test_iterated_chains_the_constraint():
    g = gg.sbm_planted(n=500, blocks=10, p_in=0.1, p_out=0.01, seed=2)
    one, r1, _ = oracle.louvain_plus_iterated(g, 1)
    plain, rp, _ = oracle.louvain_plus(g)
    assert np.array_equal(one, plain) and r1["phi"] == rp["phi"]
    three, r3, _ = oracle.louvain_plus_iterated(g, 3)
    two, _, _ = oracle.louvain_plus_constrained(g, plain)
    again, ra, _ = oracle.louvain_plus_constrained(g, two)
    assert np.array_equal(three, again) and r3["phi"] == ra["phi"]


def test_constraint_rejects_negative_labels():
    g = tiny(6, 0.5, 0)
    with pytest.raises(Exception):
        oracle.louvain_plus_constrained(g, np.array([0, 1, -1, 0, 1, 0], dtype=np.int32))


def test_uncoarsening_crosses_classes_two_cliques():
    """Two disjoint 8-cliques, constraint = vertex parity.  Coarsening can
    only form the four half-cliques (same parity, same clique), and the
    coarse graph's four vertices then have no allowed move, so coarsening
    ends after two levels.  The unconstrained uncoarsening pass at level 0
    then merges each clique: the result is the two cliques, the optimum of
    disjoint cliques."""
    src, dst = [], []
    for c in range(2):
        for i in range(8):
            for j in range(i + 1, 8):
                src.append(8 * c + i)
                dst.append(8 * c + j)
    rp, col, ew = gg.from_edges(16, np.array(src), np.array(dst))
    g = gg.modularity_inputs(rp, col, ew)
    B = (np.arange(16) % 2).astype(np.int32)
    lab, res, _ = oracle.louvain_plus_constrained(g, B, oracle.Params(uncoarsen=False))
    parts = {frozenset(np.nonzero(lab == x)[0].tolist()) for x in np.unique(lab)}
    assert parts == {frozenset(range(8 * c + b, 8 * c + 8, 2)) for c in range(2) for b in range(2)}
    assert res["levels"] == 2
    lab, res, _ = oracle.louvain_plus_constrained(g, B)
    parts = {frozenset(np.nonzero(lab == x)[0].tolist()) for x in np.unique(lab)}
    assert parts == {frozenset(range(8)), frozenset(range(8, 16))}
