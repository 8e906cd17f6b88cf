"""GPU parity of the kept tables (Section IV-A-3): the tables S(v, .) of
the vertices of degree above 256, written out by an aggregation pass and
updated in place from the movers by the following passes.  With `tables=1`
every pass after the first aggregation pass of a LocalMovePasses call
reads those vertices' argmax from the updated tables, at every level, so
the graphs below run that path through every pass, level and phase; the
results must equal the oracle's bit for bit (the oracle recomputes S from
scratch every pass, Algorithm 2).  A constructed local-move run makes a
table run out of slots and take the rebuild path."""
import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2608_01503_gb300 as lc  # noqa: E402
from tests.test_gpu_parity import check_full, compare_traces, dev, gpu_cluster, tiny_graph  # noqa: E402
from tests.test_gpu_families import FAMILIES  # noqa: E402
from tests.test_gpu_batch import run_batch  # noqa: E402

KEPT = lc.Options(tables=1)


@pytest.mark.parametrize("seed", range(40))
def test_tiny_every_pass_with_kept_tables(seed):
    check_full(tiny_graph(seed), KEPT)


def test_tiny_louvain_and_other_schedules_with_kept_tables():
    for seed in range(8):
        check_full(tiny_graph(300 + seed), lc.Options(uncoarsen=False, tables=1))
    opts = lc.Options(pass_limit=9, phi=[(1, 1), (0, 1), (1, 2)] * 3, eps=(3, 7), seed=777, tables=1)
    for seed in range(6):
        check_full(tiny_graph(400 + seed), opts)


@pytest.mark.parametrize("tables", [0, 1])
def test_mid_sized_graphs_both_modes(tables):
    opts = lc.Options(tables=tables)
    for g in (gg.sbm_planted(n=3000, blocks=30, p_in=0.03, p_out=0.002, seed=5), gg.rmat(13, seed=2),
              gg.grid_cpm(side=24)):
        res = check_full(g, opts, trace=False)
        assert (res["kernel_launches"]["table"] > 0) == (tables == 1)


def test_table_passes_run_and_match_every_pass():
    g = gg.sbm_planted(n=2000, blocks=20, p_in=0.05, p_out=0.003, seed=11)
    res = check_full(g, KEPT, trace=True)
    assert res["kernel_launches"]["table"] > 0


@pytest.mark.parametrize("name", sorted(FAMILIES))
def test_families_with_kept_tables(name):
    g = FAMILIES[name]()
    check_full(g, KEPT, trace=g.n <= 5000)


def hub_with_churning_neighbours(seed, d=260, pool=3000, m=3, extra=6000):
    """A vertex of degree d whose neighbours each touch m vertices of a random
    pool; with random starting labels, CPM 1/2 and phi = 1 the neighbours'
    clusters keep changing, and within 16 passes more than 2d distinct
    clusters have reached the hub's table (counted with the oracle's trace
    when the case was chosen: the first overflow comes at pass 4 or 5)."""
    rng = np.random.default_rng(seed)
    n = 1 + d + pool
    src = [np.zeros(d, np.int64), np.repeat(np.arange(1, d + 1), m), 1 + d + rng.integers(0, pool, extra)]
    dst = [np.arange(1, d + 1), 1 + d + rng.integers(0, pool, d * m), 1 + d + rng.integers(0, pool, extra)]
    s, t = np.concatenate(src), np.concatenate(dst)
    keep = s != t
    lo, hi = np.minimum(s[keep], t[keep]), np.maximum(s[keep], t[keep])
    key = np.unique(lo * n + hi)
    rp, col, ew = gg.from_edges(n, key // n, key % n)
    return gg.cpm_inputs(rp, col, ew, 1, 2), rng.integers(0, n, size=n).astype(np.int32)


@pytest.mark.parametrize("seed", [0, 1])
def test_overflowing_tables_are_rebuilt(seed):
    g, start = hub_with_churning_neighbours(seed)
    opts = lc.Options(pass_limit=16, phi=[(1, 1)] * 16, tables=1)
    out, res = lc.lc_local_move(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num, g.lam_den,
                                dev(start), singleton_start=False, opts=opts)
    torch.cuda.synchronize()
    C_out, phi, _ = oracle.local_move(g, start, oracle.Params(pass_limit=16, phi=[(1, 1)] * 16))
    assert np.array_equal(out.cpu().numpy(), C_out)
    assert res["phi"] == phi
    assert res["tables_rebuilt"] > 0


def test_kept_tables_with_ablations_and_symmetry_modes():
    g = gg.sbm_planted(n=1500, blocks=15, p_in=0.05, p_out=0.004, seed=3)
    for sym in (1, 2):
        check_full(g, lc.Options(symmetry=sym, phi=[(0, 1)] * 6, tables=1), trace=False)


@pytest.mark.parametrize("plus", [False, True])
def test_pleiden_with_kept_tables(plus):
    for k, g in enumerate((tiny_graph(61), tiny_graph(62), gg.rmat(12, seed=4),
                           gg.sbm_planted(n=2000, blocks=20, p_in=0.05, p_out=0.003, seed=2))):
        trace = g.n <= 100
        tr = lc.Trace() if trace else None
        labels, res = lc.lc_cluster_leiden(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num,
                                           g.lam_den, None, opts=lc.Options(uncoarsen=plus, seed=k, tables=1),
                                           trace=tr)
        torch.cuda.synchronize()
        ref, ores, oev = oracle.pleiden(g, oracle.Params(uncoarsen=plus, seed=k), trace=trace,
                                        trace_passes=trace)
        if trace:
            compare_traces(tr.events, oev)
        assert np.array_equal(labels.cpu().numpy(), ref)
        assert res["phi"] == ores["phi"] and res["levels"] == ores["levels"]


def test_constrained_with_kept_tables():
    g = gg.sbm_planted(n=1500, blocks=20, p_in=0.05, p_out=0.004, seed=8)
    prev, _, _ = oracle.louvain_plus(g)
    labels, res = lc.lc_cluster_constrained(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num,
                                            g.lam_den, dev(prev.astype(np.int32)),
                                            opts=lc.Options(tables=1))
    torch.cuda.synchronize()
    ref, ores, _ = oracle.louvain_plus_constrained(g, prev)
    assert np.array_equal(labels.cpu().numpy(), ref) and res["phi"] == ores["phi"]


def test_batch_with_kept_tables():
    graphs = [gg.rmat(9, seed=k) for k in range(3)] + [gg.sbm_planted(n=800, blocks=8, p_in=0.05,
                                                                      p_out=0.005, seed=4)]
    labels, res = run_batch(graphs, lc.Options(tables=1))
    for k, g in enumerate(graphs):
        ref, ores, _ = oracle.louvain_plus(g)
        assert np.array_equal(labels[k], ref), k
        assert res[k]["phi"] == ores["phi"], k


def test_modes_agree_on_a_larger_rmat():
    """R-MAT scale 16 (hubs of degree above 4096 keep their tables too): both
    modes give the same labels and objective."""
    g = gg.rmat(16, seed=1)
    out = [gpu_cluster(g, lc.Options(tables=t))[:2] for t in (0, 1)]
    for labels, res in out[1:]:
        assert np.array_equal(labels, out[0][0])
        assert res["phi"] == out[0][1]["phi"] and res["passes_total"] == out[0][1]["passes_total"]
    ref, ores, _ = oracle.louvain_plus(g)
    assert np.array_equal(out[0][0], ref) and out[0][1]["phi"] == ores["phi"]


def test_bad_tables_option_rejected():
    g = gg.rmat(8, seed=1)
    with pytest.raises(lc.LCError):
        gpu_cluster(g, lc.Options(tables=2))
