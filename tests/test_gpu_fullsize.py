"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (profiling on, the default schedule).  The oracle runs each whole
clustering on the host (about a minute per graph for R-MAT scale 22 and the
256^3 grid); the batched and served workloads are checked on a sample of
their graphs, each clustered alone by the oracle."""
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


def test_batched_4096_sampled():
    graphs = gg.batched_sbms(4096, seed=3)
    b = gg.pack(graphs)
    labels, res = lc.lc_cluster_batch(dev(b["row_ptr"]), dev(b["col"]), dev(b["ew"]), dev(b["vw"]),
                                      b["graph_ptr"], b["lam_num"], b["lam_den"],
                                      opts=lc.Options(profile=True))
    torch.cuda.synchronize()
    labels = labels.cpu().numpy()
    gp = b["graph_ptr"]
    # every 97th graph plus the largest one
    sample = sorted(set(range(0, 4096, 97)) | {int(np.argmax([g.nnz for g in graphs]))})
    for k in sample:
        ref, ores, _ = oracle.louvain_plus(graphs[k])
        assert np.array_equal(labels[gp[k]:gp[k + 1]], ref), k
        assert res[k]["phi"] == ores["phi"] and res[k]["n_clusters"] == ores["n_clusters"], k


def test_served_mix_sampled():
    """The served workload's largest SBM and R-MAT requests and a few small
    ones, submitted together so they share admissions."""
    params = gg.served_request_params(64, seed=4)
    graphs = gg.served_requests(64, seed=4)
    sbm = [k for k, p in enumerate(params) if p[0] == "sbm"]
    rmat = [k for k, p in enumerate(params) if p[0] == "rmat"]
    big = [max(sbm, key=lambda k: graphs[k].n), max(rmat, key=lambda k: graphs[k].n)]
    pick = big + sbm[:3] + rmat[:3]
    with lc.Server(slots=2, max_batch=8) as srv:
        ids = [srv.submit(graphs[k].row_ptr, graphs[k].col, graphs[k].ew, graphs[k].vw,
                          graphs[k].lam_num, graphs[k].lam_den) for k in pick]
        out = [srv.wait(j) for j in ids]
    for k, (labels, res, _) in zip(pick, out):
        ref, ores, _ = oracle.louvain_plus(graphs[k])
        assert np.array_equal(labels, ref), graphs[k].name
        assert res["phi"] == ores["phi"], graphs[k].name


def test_rmat22_pleiden_whole_run():
    g = gg.rmat(22, 16, seed=1, wmax=8)
    labels, res = lc.lc_cluster_leiden(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num,
                                       g.lam_den, None, opts=lc.Options(profile=True, uncoarsen=False))
    torch.cuda.synchronize()
    ref, ores, _ = oracle.pleiden(g, oracle.Params(uncoarsen=False))
    assert np.array_equal(labels.cpu().numpy(), ref)
    for k in ("phi", "n_clusters", "levels", "passes_total", "modularity"):
        assert res[k] == ores[k], k
