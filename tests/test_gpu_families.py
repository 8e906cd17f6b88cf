"""GPU parity on structured graph families: dense cliques, complete
bipartite graphs, rings and paths (deep coarsening), a star whose centre is
a hub, a barbell, heavy edge and vertex weights near the exactness guards,
and lambda at both ends of [0, 1].  Every pass, coarse graph and label is
compared with the oracle, for Louvain+ and pLeiden+."""
import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2608_01503_gb300 as lc  # noqa: E402
from tests.test_gpu_parity import check_full  # noqa: E402
from tests.test_gpu_leiden import check_leiden  # noqa: E402


def edges_graph(n, src, dst, kind="mod", lam=(1, 3), wmax=1, seed=0):
    rp, col, ew = gg.from_edges(n, np.asarray(src), np.asarray(dst), seed=seed, wmin=1, wmax=wmax)
    if kind == "mod":
        return gg.modularity_inputs(rp, col, ew)
    return gg.cpm_inputs(rp, col, ew, *lam)


def clique(n):
    i, j = np.triu_indices(n, 1)
    return edges_graph(n, i, j)


def bipartite(a, b):
    i, j = np.meshgrid(np.arange(a), a + np.arange(b), indexing="ij")
    return edges_graph(a + b, i.ravel(), j.ravel())


def ring(n, kind="cpm"):
    return edges_graph(n, np.arange(n), (np.arange(n) + 1) % n, kind=kind, lam=(1, 4))


def path(n):
    return edges_graph(n, np.arange(n - 1), np.arange(1, n), kind="cpm", lam=(1, 3))


def star(leaves):
    return edges_graph(leaves + 1, np.zeros(leaves, np.int64), np.arange(1, leaves + 1))


def barbell(k, bridge):
    """Two k-cliques joined by a path of `bridge` vertices."""
    i, j = np.triu_indices(k, 1)
    chain = np.arange(k - 1, k + bridge + 1)  # last vertex of clique 1 ... first of clique 2
    n = 2 * k + bridge
    return edges_graph(n, np.concatenate([i, i + k + bridge, chain[:-1]]),
                       np.concatenate([j, j + k + bridge, chain[1:]]))


FAMILIES = {
    "clique60": lambda: clique(60),
    "bipartite30x40": lambda: bipartite(30, 40),
    "ring5000": lambda: ring(5000),
    "ring_mod3000": lambda: ring(3000, kind="mod"),
    "path4000": lambda: path(4000),
    "star20000": lambda: star(20000),
    "barbell": lambda: barbell(25, 10),
}


@pytest.mark.parametrize("name", sorted(FAMILIES))
def test_family_louvain_plus(name):
    g = FAMILIES[name]()
    check_full(g, trace=g.n <= 5000)


@pytest.mark.parametrize("name", sorted(FAMILIES))
def test_family_pleiden_plus(name):
    g = FAMILIES[name]()
    check_leiden(g, plus=True, trace=g.n <= 5000)


def test_heavy_weights_near_the_guards():
    """Edge weights up to 2^15 (T about 2^29, Lambda T + mu V^2 about 2^59
    under modularity), and vertex weights up to 2^18 with lambda = 1/2^24."""
    rp, col, ew = gg.rmat_csr(11, 8, 0.57, 0.19, 0.19, 5, 1, 1 << 15)
    T = int(ew.astype(np.int64).sum())
    vw = gg.weighted_degree(rp, ew)
    assert T < 2**31 and T * T + int(vw.sum()) ** 2 < 2**60
    check_full(gg.Graph(rp, col, ew, vw, 1, T))
    rp2, col2, ew2 = gg.rmat_csr(11, 8, 0.57, 0.19, 0.19, 6, 1, 8)
    rng = np.random.default_rng(3)
    vw2 = rng.integers(1, 1 << 18, size=rp2.shape[0] - 1).astype(np.int64)
    check_full(gg.Graph(rp2, col2, ew2, vw2, 1, 1 << 24))


def test_epsilon_bucket_beyond_64_bits():
    """Settings inside the exactness guards where a product of the
    afterburner's bucket leaves 64 bits, so the bucket takes its 128-bit
    division: eps = 1 with eps_den = 2^31 - 1 on heavy weights (eps_den *
    delta reaches 80 bits), and CPM with lambda = 2^-40 and eps_num =
    2^31 - 1 (eps_num * Lambda reaches 71 bits).  Results still equal the
    oracle's, whose bucket is always 128-bit."""
    rp, col, ew = gg.rmat_csr(11, 8, 0.57, 0.19, 0.19, 5, 1, 1 << 15)
    T = int(ew.astype(np.int64).sum())
    check_full(gg.Graph(rp, col, ew, gg.weighted_degree(rp, ew), 1, T), lc.Options(eps=(2**31 - 1, 2**31 - 1)))
    rp2, col2, ew2 = gg.random_graph(300, 0.05, 3, wmax=4)
    check_full(gg.cpm_inputs(rp2, col2, ew2, 1, 2**40), lc.Options(eps=(2**31 - 1, 3)))


@pytest.mark.parametrize("lam", [(0, 7), (7, 7), (1, 10**9)])
def test_lambda_extremes(lam):
    rp, col, ew = gg.rmat_csr(12, 8, 0.57, 0.19, 0.19, 9, 1, 4)
    g = gg.cpm_inputs(rp, col, ew, *lam)
    check_full(g)
    check_leiden(g, plus=False, trace=False)
