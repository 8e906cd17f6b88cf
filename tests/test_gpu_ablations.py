"""GPU parity of the ablation settings of Section VI against the oracle:
no symmetry breaking, the minimum label heuristic in odd passes, phi = 0,
Louvain without uncoarsening and twice the passes; every pass traced on
tiny graphs, whole runs on larger ones."""
import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2608_01503_gb300 as lc  # noqa: E402
from tests.test_gpu_parity import check_full, tiny_graph  # noqa: E402

PHI0 = [(0, 1)] * 6
SETTINGS = {
    "none_phi0": dict(symmetry=1, phi=PHI0),
    "mlh_phi0": dict(symmetry=2, phi=PHI0),
    "phi0": dict(phi=PHI0),
    "louvain": dict(uncoarsen=False),
    "louvain_2x": dict(uncoarsen=False, pass_limit=12, phi=[(3, 4)] * 8 + [(1, 4)] * 4),
}


def _oracle_check(g, opts):
    labels, res = lc.lc_cluster(*(torch.from_numpy(np.ascontiguousarray(a)).cuda()
                                  for a in (g.row_ptr, g.col, g.ew, g.vw)), g.lam_num, g.lam_den, opts=opts)
    torch.cuda.synchronize()
    ref, ores, _ = oracle.louvain_plus(g, oracle.Params(pass_limit=opts.pass_limit, phi=opts.phi,
                                                        uncoarsen=opts.uncoarsen, symmetry=opts.symmetry))
    assert np.array_equal(labels.cpu().numpy(), ref)
    assert res["phi"] == ores["phi"] and res["passes_total"] == ores["passes_total"]


@pytest.mark.parametrize("name", sorted(SETTINGS))
@pytest.mark.parametrize("seed", range(8))
def test_tiny_every_pass(name, seed):
    check_full(tiny_graph(300 + seed), lc.Options(**SETTINGS[name]))


@pytest.mark.parametrize("name", sorted(SETTINGS))
def test_sbm_and_rmat(name):
    opts = lc.Options(**SETTINGS[name])
    for g in (gg.sbm_planted(n=4000, blocks=40, p_in=0.03, p_out=0.002, seed=6), gg.rmat(14, seed=5)):
        _oracle_check(g, opts)


def test_single_edge_swap():
    rp, col, ew = gg.from_edges(2, np.array([0]), np.array([1]))
    g = gg.modularity_inputs(rp, col, ew)
    out = {}
    for sym in (0, 1, 2):
        opts = lc.Options(symmetry=sym, phi=PHI0)
        labels, res = lc.lc_cluster(*(torch.from_numpy(np.ascontiguousarray(a)).cuda()
                                      for a in (g.row_ptr, g.col, g.ew, g.vw)), g.lam_num, g.lam_den,
                                    opts=opts)
        out[sym] = res["n_clusters"]
    assert out == {0: 1, 1: 2, 2: 1}


def test_bad_symmetry_rejected():
    g = tiny_graph(1)
    with pytest.raises(lc.LCError):
        lc.lc_cluster(*(torch.from_numpy(np.ascontiguousarray(a)).cuda()
                        for a in (g.row_ptr, g.col, g.ew, g.vw)), g.lam_num, g.lam_den,
                      opts=lc.Options(symmetry=5))
