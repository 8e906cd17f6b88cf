"""The allocation-free objective entry point (lc_objective_static) against the
regular one (lc_objective).

lc_objective_static exists for callers that cannot allocate device memory at
the point where they need the objective: an application whose memory pool
already holds the whole GPU, or a latency-bound service that forbids
cudaMalloc/cudaFree after start-up.  It keeps its scratch in one fixed array
inside the library, so this test checks, through the C ABI, that two calls in
a row (the second one reusing the array the first one left behind) give
exactly what lc_objective gives and what the CPU oracle computes from Eq. 1,
and that a graph above the array's vertex limit, labels outside [0, n), a
malformed CSR and inputs beyond the exactness guards are refused.  This file
is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle

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


def check_oracle(g, labels, got):
    """The exact objective of Eq. 1 from the CPU oracle, and the label count."""
    assert got["phi"] == oracle.objective(g, labels)
    assert got["n_clusters"] == len(np.unique(labels))


def static_rc(g, labels, rp=None, col=None, lam=None):
    """Return code of one lc_objective_static call through the C ABI."""
    lib = lc.load()
    t_rp, t_col, t_ew, t_vw, t_lab = (dev(g.row_ptr if rp is None else rp), dev(g.col if col is None else col),
                                      dev(g.ew), dev(g.vw), dev(labels))
    csr = lc._Csr(g.n, g.nnz, t_rp.data_ptr(), t_col.data_ptr() if g.nnz else None)
    res = lc._Result()
    mu, Lam = lam if lam else (g.lam_num, g.lam_den)
    rc = lib.lc_objective_static(ctypes.byref(csr), ctypes.c_void_p(t_vw.data_ptr()),
                                 ctypes.c_void_p(t_ew.data_ptr() if g.nnz else None), mu, Lam,
                                 ctypes.c_void_p(t_lab.data_ptr()), None, ctypes.byref(res))
    torch.cuda.synchronize()
    return rc


def test_two_calls_in_a_row_match_lc_objective():
    g = gg.rmat(14, seed=5)
    first = gg.random_labels(g.n, 50, 1)
    second = gg.random_labels(g.n, 3000, 2)  # more labels than the first call used
    for lab in (first, second):
        ref, got = both(g, lab)
        same(ref, got)
        check_oracle(g, lab, got)
    h = gg.grid_cpm(side=20)
    for lab in (gg.random_labels(h.n, 40, 3), np.arange(h.n, dtype=np.int32)):
        ref, got = both(h, lab)
        same(ref, got)
        check_oracle(h, lab, got)


def test_edgeless_graph():
    """No edges (T = 0): the objective is only the -mu sum of W(X)^2 - w^2 term
    and the modularity is reported as 0."""
    n = 50
    g = gg.Graph(np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32),
                 np.arange(1, n + 1, dtype=np.int64), 1, 3)
    lab = gg.random_labels(n, 7, 4)
    got = lc.lc_objective_static(dev(g.row_ptr), torch.zeros(0, dtype=torch.int32, device=DEV),
                                 torch.zeros(0, dtype=torch.int32, device=DEV), dev(g.vw), g.lam_num,
                                 g.lam_den, dev(lab))
    check_oracle(g, lab, got)
    assert got["phi"] < 0 and got["modularity"] == 0.0


def test_refuses_bad_labels_malformed_csr_and_overflow():
    g = gg.rmat(10, seed=6)
    good = gg.random_labels(g.n, 20, 5)
    assert static_rc(g, good) == 0
    bad = good.copy()
    bad[3] = g.n  # outside [0, n)
    assert static_rc(g, bad) == 1
    bad[3] = -1
    assert static_rc(g, bad) == 1
    rp = g.row_ptr.copy()
    rp[-1] -= 1  # row_ptr[n] != nnz
    assert static_rc(g, good, rp=rp) == 1
    rp = g.row_ptr.copy()
    rp[0] = 1  # row_ptr[0] != 0
    assert static_rc(g, good, rp=rp) == 1
    rp = g.row_ptr.copy()
    k = int(np.nonzero(np.diff(rp) > 1)[0][0]) + 1
    rp[k] = g.nnz + 5  # a row reaching past nnz: refused, never read
    assert static_rc(g, good, rp=rp) == 1
    col = g.col.copy()
    col[7] = g.n + 3  # a column outside [0, n): refused, never followed
    assert static_rc(g, good, col=col) == 1
    # the same call still works after the refusals (the array is cleared per call)
    assert static_rc(g, good) == 0
    # beyond the exactness guards: sum of vertex weights V with mu V^2 >= 2^60
    big = gg.Graph(g.row_ptr, g.col, g.ew, np.full(g.n, 1 << 29, np.int64), 1, 1)
    assert static_rc(big, good) == 6  # LC_ERR_OVERFLOW


def test_rejects_graphs_above_the_vertex_limit():
    lib = lc.load()
    limit = lc.lc_objective_static_max_vertices()
    assert limit == 4194304
    csr = lc._Csr(limit + 1, 0, None, None)
    res = lc._Result()
    rc = lib.lc_objective_static(ctypes.byref(csr), None, None, 1, 2, None, None, ctypes.byref(res))
    assert rc == 1 and res.error_detail == limit  # LC_ERR_ARG, nothing launched
