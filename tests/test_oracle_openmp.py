"""The oracle's OpenMP build (the all-core CPU baseline) computes exactly what
the sequential build computes: every pass, every LocalMovePasses result,
every coarse graph and the final labels, on Louvain+, Louvain, constrained
Louvain+ and pLeiden+.  Its loops over vertices and clusters write only
their own entries and sum integers, so nothing may differ."""
import os

import numpy as np
import pytest

import graphgen as gg
import oracle


def _same_events(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert x.keys() == y.keys()
        for k in x:
            if isinstance(x[k], np.ndarray):
                assert np.array_equal(x[k], y[k]), (x["kind"], x["level"], k)
            else:
                assert x[k] == y[k], (x["kind"], x["level"], k)


def _graphs():
    rp, col, ew = gg.random_graph(300, 0.03, 11, wmax=5)
    return [gg.rmat(13, seed=4), gg.sbm_planted(n=2000, blocks=20, p_in=0.05, p_out=0.002, seed=2),
            gg.grid_cpm(side=12), gg.cpm_inputs(rp, col, ew, 1, 9)]


@pytest.fixture(scope="module", autouse=True)
def threads():
    # more threads than this host has cores is fine: the results must not move
    old = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "4"
    yield
    if old is None:
        os.environ.pop("OMP_NUM_THREADS", None)
    else:
        os.environ["OMP_NUM_THREADS"] = old


@pytest.mark.parametrize("gi", range(4))
def test_openmp_build_traces_identical(gi):
    g = _graphs()[gi]
    for params in (oracle.Params(), oracle.Params(uncoarsen=False)):
        seq = oracle.louvain_plus(g, params, trace=True, trace_passes=True)
        with oracle.all_cores():
            par = oracle.louvain_plus(g, params, trace=True, trace_passes=True)
        assert np.array_equal(seq[0], par[0]) and seq[1] == par[1]
        _same_events(seq[2], par[2])


@pytest.mark.parametrize("gi", range(4))
def test_openmp_build_constrained_and_pleiden(gi):
    g = _graphs()[gi]
    B = gg.random_labels(g.n, 5, gi)
    seq_c = oracle.louvain_plus_constrained(g, B)
    seq_l = oracle.pleiden(g, trace=True)
    with oracle.all_cores():
        par_c = oracle.louvain_plus_constrained(g, B)
        par_l = oracle.pleiden(g, trace=True)
    assert np.array_equal(seq_c[0], par_c[0]) and seq_c[1] == par_c[1]
    assert np.array_equal(seq_l[0], par_l[0]) and seq_l[1] == par_l[1]
    _same_events(seq_l[2], par_l[2])
