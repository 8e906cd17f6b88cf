"""GPU parity of constrained and iterated Louvain+ (Section V-B) against the
oracle, which applies the constraint by its definition while the CUDA path
runs the coarsening passes on the graph without inter-class edges.  Labels,
every pass, every coarse graph and the exact objective must match bit for
bit."""
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


def check_constrained(g, B, opts=None, trace=True):
    tr = lc.Trace() if trace else None
    labels, res = lc.lc_cluster_constrained(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw),
                                            g.lam_num, g.lam_den, dev(B.astype(np.int32)),
                                            opts=opts, trace=tr)
    torch.cuda.synchronize()
    params = oracle.Params() if opts is None else oracle.Params(uncoarsen=opts.uncoarsen)
    ref, ores, oev = oracle.louvain_plus_constrained(g, B, params, trace=trace, trace_passes=trace)
    if trace:
        compare_traces(tr.events, oev)
    assert np.array_equal(labels.cpu().numpy(), ref)
    for k in ("phi", "n_clusters", "levels", "passes_total", "objective", "modularity"):
        assert res[k] == ores[k], k
    return res


@pytest.mark.parametrize("seed", range(24))
def test_tiny_constrained_every_pass(seed):
    g = tiny_graph(seed)
    rng = np.random.default_rng(seed + 500)
    B = rng.integers(0, int(rng.integers(1, 5)), size=g.n).astype(np.int32)
    check_constrained(g, B)


def test_constraint_is_a_previous_clustering():
    for seed in range(4):
        g = gg.sbm_planted(n=1500, blocks=20, p_in=0.05, p_out=0.004, seed=seed)
        prev, _, _ = oracle.louvain_plus(g)
        check_constrained(g, prev)
        check_constrained(g, prev, lc.Options(uncoarsen=False))


def test_special_constraints():
    g = gg.rmat(11, seed=4)
    check_constrained(g, np.zeros(g.n, dtype=np.int32), trace=False)
    res = check_constrained(g, np.arange(g.n, dtype=np.int32), trace=False)
    assert res["levels"] == 1
    # large label values only matter through equality
    B = (np.arange(g.n) % 3).astype(np.int32) * 700_000_001
    check_constrained(g, B, trace=False)


def test_rmat_constrained_by_its_own_clustering():
    g = gg.rmat(15, seed=7)
    prev, _, _ = oracle.louvain_plus(g)
    check_constrained(g, prev, trace=False)


@pytest.mark.parametrize("iterations", [1, 2, 4])
def test_iterated_equals_oracle(iterations):
    g = gg.sbm_planted(n=3000, blocks=30, p_in=0.03, p_out=0.002, seed=9)
    labels, res = lc.lc_cluster_iterated(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num,
                                         g.lam_den, iterations)
    torch.cuda.synchronize()
    ref, ores, _ = oracle.louvain_plus_iterated(g, iterations)
    assert np.array_equal(labels.cpu().numpy(), ref)
    for k in ("phi", "n_clusters", "levels", "passes_total", "modularity"):
        assert res[k] == ores[k], k


def test_iterated_rejects_zero_iterations():
    g = gg.rmat(8, seed=1)
    with pytest.raises(lc.LCError):
        lc.lc_cluster_iterated(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num,
                               g.lam_den, 0)


def test_degenerate_graphs():
    rp, col, ew = gg.from_edges(2, np.array([0]), np.array([1]))
    g = gg.modularity_inputs(rp, col, ew)
    check_constrained(g, np.array([0, 0], dtype=np.int32))
    check_constrained(g, np.array([0, 1], dtype=np.int32))
    e = gg.cpm_inputs(np.zeros(5, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32), 1, 3)
    check_constrained(e, np.zeros(4, dtype=np.int32))
