"""The allocation-free objective entry point (lc_objective_static) against the
regular one (lc_objective).

lc_objective_static exists for callers that cannot allocate device memory at
the point where they need the objective: an application whose memory pool
already holds the whole GPU, or a latency-bound service that forbids
cudaMalloc/cudaFree after start-up.  It keeps its scratch in one fixed array
inside the library, so this test checks, through the C ABI, that two calls in
a row (the second one reusing the array the first one left behind) give
exactly what lc_objective gives, and that a graph above the array's vertex
limit is refused.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2608_01503_gb300 as lc  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def both(g, labels):
    args = (dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num, g.lam_den, dev(labels))
    ref = lc.lc_objective(*args)
    got = lc.lc_objective_static(*args)
    torch.cuda.synchronize()
    return ref, got


def same(ref, got):
    # integer results are exact; the FP64 views come from the same integers
    assert got["phi"] == ref["phi"]
    assert got["n_clusters"] == ref["n_clusters"]
    assert got["objective"] == ref["objective"]
    assert got["modularity"] == ref["modularity"]


def test_two_calls_in_a_row_match_lc_objective():
    g = gg.rmat(14, seed=5)
    first = gg.random_labels(g.n, 50, 1)
    second = gg.random_labels(g.n, 3000, 2)  # more labels than the first call used
    same(*both(g, first))
    same(*both(g, second))
    h = gg.grid_cpm(side=20)
    same(*both(h, gg.random_labels(h.n, 40, 3)))
    same(*both(h, np.arange(h.n, dtype=np.int32)))


def test_rejects_graphs_above_the_vertex_limit():
    lib = lc.load()
    limit = lc.lc_objective_static_max_vertices()
    assert limit == 4194304
    csr = lc._Csr(limit + 1, 0, None, None)
    res = lc._Result()
    rc = lib.lc_objective_static(ctypes.byref(csr), None, None, 1, 2, None, None, ctypes.byref(res))
    assert rc == 1 and res.error_detail == limit  # LC_ERR_ARG, nothing launched
