"""Pins of Algorithm 1's coarsening loop in the CPU oracle: when it stops,
and how it renumbers labels between levels.

Algorithm 1 coarsens while the level's LocalMovePasses call merged
something: a level whose call returns all singletons (|C_l| = |V_l|) is the
last.  Every check below re-derives what the loop must have done from the
oracle's trace with tools other than the loop itself:

* LocalMovePasses from singletons on every traced graph G_l, re-run through
  the separately pinned ``oracle.local_move`` (test_oracle_pins.py), must
  merge something on every level but the last and nothing on the last;
* each coarse graph must equal the membership product P^T A P of its level
  (scipy sparse products, not the oracle's contraction);
* the dense labels handed to the contraction must number the clusters in
  ascending order of their old ids (numpy's ``unique``), and so must the
  final labels;
* the level count and the number of contractions must agree with the stop.

Plausible mistakes are planted in copies of lc_oracle.c, compiled here with
gcc: stopping while merges remain (a level that merged under half, or under
a tenth, of its vertices ends the coarsening) and running one level too many
(the stop also waits for the previous level to have merged nothing).  All
leave the final objective plausible, and all must be rejected.
"""
from __future__ import annotations

import json
import os
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

import graphgen as gg
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE_SRC = os.path.join(os.path.dirname(HERE), "oracle", "lc_oracle.c")

STOP_TEST = "if (k == n) { /* |C_l| = |V_l| */"
MUTANTS = {
    # stops as soon as a level merges fewer than half of its vertices
    "stops_early": "if (2 * k > n) { /* |C_l| = |V_l| */",
    # stops as soon as a level merges fewer than a tenth of its vertices
    "stops_on_small_merge": "if (10 * k >= 9 * n) { /* |C_l| = |V_l| */",
    # contracts one all-singleton level before stopping
    "extra_level": "if (k == n && (L == 0 || G[L - 1].n == n)) { /* |C_l| = |V_l| */",
}


def _adjacency(rp, col, ew, n):
    return sp.csr_matrix((np.asarray(ew, np.int64), np.asarray(col), np.asarray(rp)), shape=(n, n))


def _ascending_relabel(C):
    """Dense ids numbered in ascending order of the old id."""
    return np.unique(np.asarray(C), return_inverse=True)[1].astype(np.int32)


def coarsening_violations(g, params, labels, res, events) -> list:
    """Every way the traced run departs from Algorithm 1's coarsening loop."""
    bad = []
    lmp_c = {e["level"]: e for e in events if e["kind"] == "lmp" and e["phase"] == "coarsen"}
    lmp_u = {e["level"]: e for e in events if e["kind"] == "lmp" and e["phase"] == "uncoarsen"}
    con = {e["level"]: e for e in events if e["kind"] == "contract"}
    if not lmp_c:
        return ["no coarsening LocalMovePasses call traced"]
    top = max(lmp_c)
    if sorted(lmp_c) != list(range(top + 1)):
        bad.append(f"coarsening levels {sorted(lmp_c)}")
    if sorted(con) != list(range(top)):
        bad.append(f"contractions at levels {sorted(con)} for {top + 1} levels")
    if res["levels"] != top + 1:
        bad.append(f"levels {res['levels']} reported, {top + 1} traced")
    G = g
    for l in range(top + 1):
        C = lmp_c[l]["C"]
        if C.shape[0] != G.n:
            bad.append(f"level {l}: {C.shape[0]} labels for {G.n} vertices")
            break
        ref, _, _ = oracle.local_move(G, np.arange(G.n, dtype=np.int32), params)
        if not np.array_equal(C, ref):
            bad.append(f"level {l}: traced clustering is not LocalMovePasses from singletons")
        k = len(np.unique(C))
        if l < top:
            if k == G.n:
                bad.append(f"level {l} merged nothing, yet the coarsening went on")
            if l not in con:
                break
            ev = con[l]
            dense = _ascending_relabel(C)
            if not np.array_equal(ev["C"], dense):
                bad.append(f"level {l}: contraction labels not numbered by ascending old id")
            if ev["cn"] != k:
                bad.append(f"level {l}: {ev['cn']} coarse vertices for {k} clusters")
            # the coarse graph is P^T A P without its diagonal (Section III-A)
            P = sp.csr_matrix((np.ones(G.n, np.int64), (np.arange(G.n), dense)), shape=(G.n, k))
            Ac = (P.T @ _adjacency(G.row_ptr, G.col, G.ew, G.n) @ P).tolil()
            Ac.setdiag(0)
            Ac = Ac.tocsr()
            Ac.eliminate_zeros()
            got = _adjacency(ev["row_ptr"], ev["col"], ev["ew"], k)
            if (got != Ac).nnz != 0:
                bad.append(f"level {l}: coarse graph is not the membership product")
            if not np.array_equal(ev["vw"], np.bincount(dense, weights=G.vw, minlength=k).astype(np.int64)):
                bad.append(f"level {l}: coarse vertex weights")
            G = gg.Graph(ev["row_ptr"], ev["col"], ev["ew"], ev["vw"], g.lam_num, g.lam_den)
        else:
            if k != G.n:
                bad.append(f"level {l} is the last but merged {G.n - k} vertices")
            if not np.array_equal(C, np.arange(G.n)):
                bad.append(f"level {l}: an all-singleton result must be the identity labelling")
    # final labels: the level-0 result numbered by ascending old id
    if top == 0:
        final0 = lmp_c[0]["C"]
    elif params.uncoarsen:
        final0 = lmp_u[0]["C"] if 0 in lmp_u else None
    else:
        cur = np.arange(lmp_c[top]["C"].shape[0])
        for l in range(top - 1, -1, -1):
            cur = cur[con[l]["C"]]
        final0 = cur
    if final0 is None:
        bad.append("no level-0 uncoarsening result traced")
    elif not np.array_equal(labels, _ascending_relabel(final0)):
        bad.append("final labels not numbered by ascending old id")
    return bad


def _graphs():
    out = [gg.sbm_planted(n=600, blocks=6, p_in=0.08, p_out=0.004, seed=3),
           gg.sbm_planted(n=2000, blocks=20, p_in=0.05, p_out=0.002, seed=5)]
    # a ring of 4-cliques coarsens over several levels
    src, dst = [], []
    K, R = 4, 24
    for r in range(R):
        b = K * r
        for a in range(K):
            for c in range(a + 1, K):
                src.append(b + a)
                dst.append(b + c)
        src.append(b + K - 1)
        dst.append((b + K) % (K * R))
    rp, col, ew = gg.from_edges(K * R, src, dst)
    out.append(gg.modularity_inputs(rp, col, ew, name="clique_ring"))
    # the hand-derived cases of tests/golden/closed_forms.json
    with open(os.path.join(HERE, "golden", "closed_forms.json")) as f:
        for case in json.load(f)["cases"]:
            rp, col, ew = gg.from_edges(case["n"], [e[0] for e in case["edges"]],
                                        [e[1] for e in case["edges"]])
            out.append(gg.modularity_inputs(rp, col, ew, name=case["name"])
                       if case["objective"] == "modularity"
                       else gg.cpm_inputs(rp, col, ew, *case["lambda"], name=case["name"]))
    for seed in range(6):
        rp, col, ew = gg.random_graph(40, 0.08, 300 + seed, wmax=3)
        out.append(gg.modularity_inputs(rp, col, ew, name=f"gnp40_{seed}") if seed % 2 == 0
                   else gg.cpm_inputs(rp, col, ew, 1, 6, name=f"gnp40_{seed}"))
    return out


GRAPHS = _graphs()


@pytest.mark.parametrize("uncoarsen", [True, False])
@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_coarsening_stops_exactly_when_a_level_merges_nothing(gi, uncoarsen):
    g = GRAPHS[gi]
    params = oracle.Params(uncoarsen=uncoarsen)
    labels, res, events = oracle.louvain_plus(g, params, trace=True)
    assert coarsening_violations(g, params, labels, res, events) == []


def test_the_graphs_coarsen_over_several_levels():
    """The pins above are only meaningful if the runs go past level 0."""
    levels = [oracle.louvain_plus(g)[1]["levels"] for g in GRAPHS]
    assert max(levels) >= 3 and sum(lv >= 2 for lv in levels) >= 8, levels


def _build_mutant(tmp_path, name):
    src = open(ORACLE_SRC).read()
    assert src.count(STOP_TEST) == 1, "the stop test of the coarsening loop moved"
    path = tmp_path / f"lc_oracle_{name}.c"
    path.write_text(src.replace(STOP_TEST, MUTANTS[name]))
    lib = tmp_path / f"liboracle_{name}.so"
    subprocess.check_call(["gcc", *oracle.GCC_FLAGS, str(path), "-o", str(lib)])
    return str(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_stop_mistakes_are_caught(tmp_path, name):
    lib = _build_mutant(tmp_path, name)
    caught = 0
    for g in GRAPHS:
        params = oracle.Params()
        with oracle.library(lib):
            labels, res, events = oracle.louvain_plus(g, params, trace=True)
        caught += bool(coarsening_violations(g, params, labels, res, events))
    assert caught >= 2, f"planted mistake '{name}' passed the pins on {len(GRAPHS) - caught} graphs"
