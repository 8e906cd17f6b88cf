"""Host-side logic that needs no GPU: the packing of batches, the workload
recipes, option marshalling into the C structs, and the benchmark's
percentile helper."""
import ctypes
import os
import sys

import numpy as np

import graphgen as gg
import paper_2608_01503_gb300 as lc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_pack_is_the_disjoint_union():
    graphs = [gg.rmat(6, seed=k) for k in range(4)] + [gg.sbm_planted(n=50, blocks=5, p_in=0.3,
                                                                      p_out=0.02, seed=1)]
    b = gg.pack(graphs)
    gp = b["graph_ptr"]
    assert gp[0] == 0 and gp[-1] == sum(g.n for g in graphs)
    for k, g in enumerate(graphs):
        lo, hi = gp[k], gp[k + 1]
        rows = b["row_ptr"][lo:hi + 1] - b["row_ptr"][lo]
        assert np.array_equal(rows, g.row_ptr)
        e0, e1 = b["row_ptr"][lo], b["row_ptr"][hi]
        assert np.array_equal(b["col"][e0:e1] - lo, g.col)
        assert np.array_equal(b["ew"][e0:e1], g.ew)
        assert np.array_equal(b["vw"][lo:hi], g.vw)
        assert b["lam_num"][k] == g.lam_num and b["lam_den"][k] == g.lam_den


def test_batched_recipe_and_expected_edges():
    params = gg.batched_sbm_params(256, seed=3)
    ns = np.array([p[0] for p in params])
    assert ns.min() >= 100 and ns.max() <= 100_000
    graphs = gg.batched_sbms(32, seed=3, threads=2)
    for p, g in zip(gg.batched_sbm_params(32, seed=3), graphs):
        assert g.n == p[0]
        assert abs(g.nnz - gg.expected_nnz(p)) <= 6 * np.sqrt(gg.expected_nnz(p)) + 10
    sub = gg.batched_sbms(32, seed=3, threads=2, indices=[3, 17])
    assert np.array_equal(sub[1].col, graphs[17].col)


def test_served_recipe_mix():
    params = gg.served_request_params(2000, seed=4)
    kinds = [p[0] for p in params]
    frac_sbm = kinds.count("sbm") / len(kinds)
    assert 0.66 < frac_sbm < 0.74
    frac_cpm = sum(p[2] for p in params) / len(params)
    assert 0.45 < frac_cpm < 0.55
    scales = [p[1] for p in params if p[0] == "rmat"]
    assert min(scales) >= 10 and max(scales) <= 20


def test_options_marshalling():
    o = lc.Options(pass_limit=9, phi=[(1, 2)] * 9, eps=(3, 7), seed=0xFFFFFFFF + 5, uncoarsen=False,
                   validate=False, profile=True, symmetry=2, tables=1)
    c = lc._c_opts(o, ctypes.c_void_p(0))
    assert c.tables == 1
    assert c.pass_limit == 9 and (c.eps_num, c.eps_den) == (3, 7)
    assert [(c.phi_num[i], c.phi_den[i]) for i in range(9)] == [(1, 2)] * 9
    assert c.seed == 4  # 32-bit salt
    assert (c.uncoarsen, c.validate, c.profile, c.symmetry) == (0, 0, 1, 2)
    d = lc._c_opts(None, ctypes.c_void_p(0))
    assert d.pass_limit == 6 and d.symmetry == 0 and d.uncoarsen == 1 and d.tables == 0


def test_bench_percentile_helper():
    sys.path.insert(0, ROOT)
    import bench

    xs = [5, 1, 4, 2, 3]
    assert bench._pct(xs, 0.5) == 3 and bench._pct(xs, 0.99) == 5 and bench._pct([], 0.5) is None
    assert set(bench.ABLATIONS) >= {"default", "louvain", "phi0", "mlh_phi0", "no_symmetry_phi0"}


def test_tuning_cache_round_trip(tmp_path):
    """save_tuning / load_tuning keep one entry per workload and device, and
    tuned_options carries every launch setting into the options (explicit
    keywords win)."""
    import paper_2608_01503_gb300 as lc

    path = str(tmp_path / "tuning.json")
    assert lc.load_tuning("rmat22/X", path) is None
    t1 = {"bins": [8, 16, 32, 64, 256, 512, 1024, 2048, 4096], "hub_chunk": 4096,
          "ab_threads": [1, 16, 16, 128, 128], "graphs": True, "ms_best": 1.0, "ms_default": 2.0, "trials": 3}
    t2 = dict(t1, hub_chunk=2048, graphs=False)
    lc.save_tuning("rmat22/X", t1, path)
    lc.save_tuning("batched/X", t2, path)
    assert lc.load_tuning("rmat22/X", path) == t1 and lc.load_tuning("batched/X", path) == t2
    o = lc.tuned_options(t1, profile=True)
    assert o.bins == tuple(t1["bins"]) and o.hub_chunk == 4096 and o.graphs is True
    assert o.ab_threads == tuple(t1["ab_threads"]) and o.profile is True
    assert lc.tuned_options(t1, graphs=False).graphs is False
    assert lc.tuned_options(None) == lc.Options()
