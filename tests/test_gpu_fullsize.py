"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (profiling on, the default schedule).  The oracle runs each whole
clustering on the host (about a minute per graph for R-MAT scale 22 and the
256^3 grid); every graph of the batched workload and of the served
workload's request pool is clustered alone by the oracle, the graphs spread
over the host's cores."""
import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2608_01503_gb300 as lc  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def check_whole(g):
    labels, res = lc.lc_cluster(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num,
                                g.lam_den, opts=lc.Options(profile=True))
    torch.cuda.synchronize()
    ref, ores, _ = oracle.louvain_plus(g)
    assert np.array_equal(labels.cpu().numpy(), ref)
    for k in ("phi", "n_clusters", "levels", "passes_total", "modularity"):
        assert res[k] == ores[k], k


def test_rmat22_whole_run():
    check_whole(gg.rmat(22, 16, seed=1, wmax=8))


def test_grid256_whole_run():
    check_whole(gg.grid_cpm(side=256))


def test_batched_4096_every_graph():
    graphs = gg.batched_sbms(4096, seed=3)
    b = gg.pack(graphs)
    labels, res = lc.lc_cluster_batch(dev(b["row_ptr"]), dev(b["col"]), dev(b["ew"]), dev(b["vw"]),
                                      b["graph_ptr"], b["lam_num"], b["lam_den"],
                                      opts=lc.Options(profile=True))
    torch.cuda.synchronize()
    labels = labels.cpu().numpy()
    gp = b["graph_ptr"]
    refs = oracle.louvain_plus_many(graphs)
    for k, (ref, ores) in enumerate(refs):
        assert np.array_equal(labels[gp[k]:gp[k + 1]], ref), k
        for key in ("phi", "n_clusters", "levels", "modularity"):
            assert res[k][key] == ores[key], (k, key)


def test_served_pool_every_request():
    """The served workload's whole 64-graph request pool, submitted together
    so that requests share admissions and slots overlap on the device."""
    graphs = gg.served_requests(64, seed=4)
    with lc.Server(slots=4, max_batch=8) as srv:
        ids = [srv.submit(g.row_ptr, g.col, g.ew, g.vw, g.lam_num, g.lam_den) for g in graphs]
        out = [srv.wait(j) for j in ids]
    refs = oracle.louvain_plus_many(graphs)
    for g, (labels, res, _), (ref, ores) in zip(graphs, out, refs):
        assert np.array_equal(labels, ref), g.name
        for key in ("phi", "n_clusters", "levels", "modularity"):
            assert res[key] == ores[key], (g.name, key)


def test_rmat22_pleiden_whole_run():
    g = gg.rmat(22, 16, seed=1, wmax=8)
    labels, res = lc.lc_cluster_leiden(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num,
                                       g.lam_den, None, opts=lc.Options(profile=True, uncoarsen=False))
    torch.cuda.synchronize()
    ref, ores, _ = oracle.pleiden(g, oracle.Params(uncoarsen=False))
    assert np.array_equal(labels.cpu().numpy(), ref)
    for k in ("phi", "n_clusters", "levels", "passes_total", "modularity"):
        assert res[k] == ores[k], k
