"""GPU parity of pLeiden / pLeiden+ (Section V) against the oracle: every
pass, every LocalMovePasses result, every coarse graph (contracted on the
refinement) and the final labels and objective, bit for bit."""
import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2608_01503_gb300 as lc  # noqa: E402
from tests.test_gpu_parity import compare_traces, dev, tiny_graph  # noqa: E402


def check_leiden(g, plus, initial=None, trace=True, seed=0):
    tr = lc.Trace() if trace else None
    opts = lc.Options(uncoarsen=plus, seed=seed)
    labels, res = lc.lc_cluster_leiden(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num,
                                       g.lam_den, None if initial is None else dev(initial.astype(np.int32)),
                                       opts=opts, trace=tr)
    torch.cuda.synchronize()
    ref, ores, oev = oracle.pleiden(g, oracle.Params(uncoarsen=plus, seed=seed), C_in=initial,
                                    trace=trace, trace_passes=trace)
    if trace:
        compare_traces(tr.events, oev)
    assert np.array_equal(labels.cpu().numpy(), ref)
    for k in ("phi", "n_clusters", "levels", "passes_total", "objective", "modularity"):
        assert res[k] == ores[k], k
    return ref, res


@pytest.mark.parametrize("seed", range(32))
def test_tiny_every_pass(seed):
    check_leiden(tiny_graph(seed), plus=bool(seed % 2), seed=seed % 5)


@pytest.mark.parametrize("plus", [False, True])
def test_sbm_and_rmat(plus):
    for g in (gg.sbm_planted(n=3000, blocks=30, p_in=0.03, p_out=0.002, seed=5), gg.rmat(13, seed=2)):
        check_leiden(g, plus)


def test_initial_clustering_and_local_move_alt():
    """Feeding pLeiden its own output makes the first LocalMovePasses call
    find nothing, so LocalMoveAlt runs; random starting labels too."""
    for seed in range(6):
        g = tiny_graph(200 + seed)
        lab, _ = check_leiden(g, plus=False)
        check_leiden(g, plus=False, initial=lab)
        check_leiden(g, plus=True, initial=gg.random_labels(g.n, max(1, g.n // 4), seed))
    g = gg.sbm_planted(n=2000, blocks=20, p_in=0.05, p_out=0.003, seed=7)
    lab, _ = check_leiden(g, plus=False, trace=False)
    check_leiden(g, plus=False, initial=lab, trace=False)


def test_rmat16_and_grid():
    check_leiden(gg.rmat(16, seed=3), plus=True, trace=False)
    check_leiden(gg.grid_cpm(side=20), plus=False, trace=False)


def test_rejects_initial_labels_out_of_range():
    g = gg.rmat(8, seed=1)
    bad = np.full(g.n, g.n, dtype=np.int32)
    with pytest.raises(lc.LCError):
        lc.lc_cluster_leiden(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num, g.lam_den,
                             dev(bad))


@pytest.mark.parametrize("plus", [False, True])
def test_degenerate_graphs(plus):
    """Single vertex, edgeless graph, one edge, a star."""
    cases = [gg.cpm_inputs(np.zeros(2, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32), 1, 2),
             gg.cpm_inputs(np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32), 1, 2)]
    rp, col, ew = gg.from_edges(2, np.array([0]), np.array([1]))
    cases.append(gg.modularity_inputs(rp, col, ew))
    rp, col, ew = gg.from_edges(40, np.zeros(39, np.int64), np.arange(1, 40))
    cases.append(gg.modularity_inputs(rp, col, ew))
    for g in cases:
        check_leiden(g, plus)


def test_empty_graph():
    g = gg.cpm_inputs(np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32), 1, 2)
    labels, res = lc.lc_cluster_leiden(dev(g.row_ptr), torch.zeros(0, dtype=torch.int32, device="cuda"),
                                       torch.zeros(0, dtype=torch.int32, device="cuda"),
                                       torch.zeros(0, dtype=torch.int64, device="cuda"), 1, 2)
    assert labels.numel() == 0 and res["n_clusters"] == 0
