"""Pins of the oracle's symmetry-breaking ablations (Section VI's ablation
study): no filter (every candidate moves) and the minimum label heuristic
(MLH) in odd passes.

* Every pass is checked against the definition and Eq. 1: the movers are
  the candidates, minus (MLH, odd passes) a singleton joining a singleton
  cluster with a larger label; the update applies exactly those moves and
  Phi after the pass is the pair objective.
* The destructive interaction the paper describes, closed form: on a single
  edge both endpoints want to join each other.  Without symmetry breaking
  they swap forever and the result stays two singletons; MLH lets only the
  larger label move, and the afterburner only the earlier one: one cluster.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from tests import brute
from tests.test_oracle_pins import CASES, tiny


@pytest.mark.parametrize("symmetry", [1, 2])
@pytest.mark.parametrize("n,p,seed,lam", CASES)
def test_pass_movers_by_definition(symmetry, n, p, seed, lam):
    g = tiny(n, p, seed, lam=lam)
    A = brute.dense(g.row_ptr, g.col, g.ew)
    P = brute.pair_matrix(A, g.vw, g.lam_num, g.lam_den)
    params = oracle.Params(symmetry=symmetry, phi=[(0, 1)] * 6)
    for start in (np.arange(n, dtype=np.int32), gg.random_labels(n, 3, seed + 5)):
        _, _, events = oracle.local_move(g, start, params, trace=True)
        for ev in events:
            if ev["kind"] != "pass":
                continue
            C, D, L = ev["C_before"], ev["D"], ev["in_L"]
            size = np.bincount(C, minlength=n)
            expect = L.copy()
            if symmetry == 2 and ev["pass"] % 2 == 1:
                for v in range(n):
                    if L[v] and size[C[v]] == 1 and D[v] >= 0 and size[D[v]] == 1 and D[v] > C[v]:
                        expect[v] = False
            assert np.array_equal(ev["in_M"], expect), (ev["pass"],)
            Ca = ev["C"]
            for v in range(n):
                if expect[v] and D[v] >= 0:
                    assert Ca[v] == D[v]
                elif expect[v]:
                    assert np.sum(Ca == Ca[v]) == 1
                else:
                    assert Ca[v] == C[v]
            assert ev["phi"] == brute.pair_objective(P, Ca)


def test_single_edge_swap_closed_form():
    rp, col, ew = gg.from_edges(2, np.array([0]), np.array([1]))
    g = gg.modularity_inputs(rp, col, ew)  # w(v) = 1, lambda = 1/2
    phi0 = [(0, 1)] * 6
    lab, res, _ = oracle.louvain_plus(g, oracle.Params(symmetry=1, phi=phi0))
    assert res["n_clusters"] == 2 and res["phi"] == 0  # the two vertices swap every pass
    for sym in (0, 2):
        lab, res, _ = oracle.louvain_plus(g, oracle.Params(symmetry=sym, phi=phi0))
        # one cluster: Phi = Lambda * (2 w(u,v) - 2 lambda w(u) w(v)) = 2 * (2 - 1) = 2
        assert res["n_clusters"] == 1 and res["phi"] == 2


def test_bad_symmetry_rejected():
    g = tiny(6, 0.5, 0)
    with pytest.raises(Exception):
        oracle.louvain_plus(g, oracle.Params(symmetry=3))
