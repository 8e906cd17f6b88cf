"""Batched form: many graphs packed into one CSR and clustered together must
give every graph exactly the result it gets alone (and the oracle's)."""
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


def mixed_graphs(seed=0):
    rng = np.random.default_rng(seed)
    graphs = []
    for k in range(18):
        kind = k % 6
        if kind == 0:
            rp, col, ew = gg.random_graph(int(rng.integers(2, 60)), 0.2, seed * 100 + k, wmax=5)
            graphs.append(gg.modularity_inputs(rp, col, ew))
        elif kind == 1:
            graphs.append(gg.sbm_planted(n=int(rng.integers(200, 2000)), blocks=int(rng.integers(2, 20)),
                                         p_in=0.1, p_out=0.005, seed=k))
        elif kind == 2:
            graphs.append(gg.rmat(int(rng.integers(8, 12)), seed=k))
        elif kind == 3:
            rp, col, ew = gg.grid3d_csr(6, 7, 5, 0.05, k, 1, 9)
            graphs.append(gg.cpm_inputs(rp, col, ew, 1, int(rng.integers(3, 40))))
        elif kind == 4:
            rp, col, ew = gg.random_graph(int(rng.integers(20, 80)), 0.1, seed * 100 + k, wmax=3)
            vw = rng.integers(1, 5, size=rp.shape[0] - 1).astype(np.int64)
            graphs.append(gg.Graph(rp, col, ew, vw, int(rng.integers(0, 4)), 17))
        else:
            n = int(rng.integers(1, 5))
            rp, col, ew = gg.from_edges(n, [], [])
            graphs.append(gg.cpm_inputs(rp, col, ew, 1, 3))  # edgeless
    return graphs


def run_batch(graphs, opts=None):
    b = gg.pack(graphs)
    labels, res = lc.lc_cluster_batch(dev(b["row_ptr"]), dev(b["col"]), dev(b["ew"]), dev(b["vw"]),
                                      b["graph_ptr"], b["lam_num"], b["lam_den"], opts=opts)
    torch.cuda.synchronize()
    lab = labels.cpu().numpy()
    gp = b["graph_ptr"]
    return [lab[gp[k]:gp[k + 1]] for k in range(len(graphs))], res


def single(g, opts=None):
    labels, res = lc.lc_cluster(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num, g.lam_den,
                                opts=opts)
    return labels.cpu().numpy(), res


@pytest.mark.parametrize("seed", [0, 1])
def test_batch_matches_single_and_oracle(seed):
    graphs = mixed_graphs(seed)
    labels, res = run_batch(graphs)
    for k, g in enumerate(graphs):
        ref, ores, _ = oracle.louvain_plus(g)
        assert np.array_equal(labels[k], ref), k
        assert res[k]["phi"] == ores["phi"], k
        assert res[k]["n_clusters"] == ores["n_clusters"], k
        assert res[k]["levels"] == ores["levels"], k
        assert res[k]["passes_total"] == ores["passes_total"], k
        assert res[k]["modularity"] == ores["modularity"], k
        assert res[k]["objective"] == ores["objective"], k
        one, r1 = single(g)
        assert np.array_equal(one, labels[k]) and r1["phi"] == res[k]["phi"], k


def test_batch_without_uncoarsening_and_order_independence():
    graphs = mixed_graphs(2)
    opts = lc.Options(uncoarsen=False)
    a, ra = run_batch(graphs, opts)
    b, rb = run_batch(graphs[::-1], opts)
    for k, g in enumerate(graphs):
        ref, ores, _ = oracle.louvain_plus(g, oracle.Params(uncoarsen=False))
        assert np.array_equal(a[k], ref)
        assert np.array_equal(b[len(graphs) - 1 - k], ref)
        assert ra[k]["phi"] == ores["phi"] == rb[len(graphs) - 1 - k]["phi"]


def test_batch_of_one_and_empty_members():
    g = gg.sbm_planted(n=800, blocks=8, seed=4)
    rp, col, ew = gg.from_edges(0, [], [])
    empty = gg.cpm_inputs(rp, col, ew, 1, 2)
    labels, res = run_batch([g])
    ref, ores, _ = oracle.louvain_plus(g)
    assert np.array_equal(labels[0], ref) and res[0]["phi"] == ores["phi"]
    labels, res = run_batch([empty, g, empty])
    assert labels[0].size == 0 and labels[2].size == 0 and res[0]["n_clusters"] == 0
    assert np.array_equal(labels[1], ref) and res[1]["phi"] == ores["phi"]


def test_batch_rejects_edges_across_graphs():
    graphs = [gg.sbm_planted(n=100, blocks=2, seed=1), gg.sbm_planted(n=100, blocks=2, seed=2)]
    b = gg.pack(graphs)
    gp = b["graph_ptr"].copy()
    gp[1] = 90  # ranges no longer match the edges
    with pytest.raises(lc.LCError) as ei:
        lc.lc_cluster_batch(dev(b["row_ptr"]), dev(b["col"]), dev(b["ew"]), dev(b["vw"]), gp,
                            b["lam_num"], b["lam_den"])
    assert ei.value.code == 1
