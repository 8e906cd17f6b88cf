"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs.  Integer results (labels, destinations, survivors,
coarse graphs, the exact objective) must match bit for bit; the FP64
objective and modularity are computed from the same exact integers and must
be identical."""
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


def gpu_cluster(g, opts=None, trace=False):
    tr = lc.Trace() if trace else None
    labels, res = lc.lc_cluster(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num,
                                g.lam_den, opts=opts, trace=tr)
    torch.cuda.synchronize()
    return labels.cpu().numpy(), res, (tr.events if tr else None)


def oracle_params(opts):
    if opts is None:
        return oracle.Params()
    return oracle.Params(pass_limit=opts.pass_limit, phi=opts.phi, eps=opts.eps, seed=opts.seed,
                         uncoarsen=opts.uncoarsen, symmetry=opts.symmetry)


def compare_traces(gpu_ev, orc_ev):
    gp = [e for e in gpu_ev if e["kind"] == "pass"]
    op = [e for e in orc_ev if e["kind"] == "pass"]
    assert len(gp) == len(op), (len(gp), len(op))
    for a, b in zip(gp, op):
        where = (b["level"], b["phase"], b["pass"])
        assert (a["level"], a["phase"], a["pass"]) == where
        inL = b["in_L"]
        assert np.array_equal(a["D"] != -1, inL), where
        assert np.array_equal(a["D"][inL], b["D"][inL]), where
        assert np.array_equal(a["in_M"], b["in_M"]), where
        assert np.array_equal(a["C"], b["C"]), where
        assert a["phi"] == b["phi"], where
        assert a["count_L"] == b["count_L"] and a["count_M"] == b["count_M"], where
    gl = [e for e in gpu_ev if e["kind"] == "lmp"]
    ol = [e for e in orc_ev if e["kind"] == "lmp"]
    assert len(gl) == len(ol)
    for a, b in zip(gl, ol):
        assert np.array_equal(a["C"], b["C"]) and a["phi"] == b["phi"], (b["level"], b["phase"])
    gc = [e for e in gpu_ev if e["kind"] == "contract"]
    oc = [e for e in orc_ev if e["kind"] == "contract"]
    assert len(gc) == len(oc)
    for a, b in zip(gc, oc):
        assert np.array_equal(a["C"], b["C"])
        assert_same_graph((a["row_ptr"], a["col"], a["ew"], a["vw"]),
                          (b["row_ptr"], b["col"], b["ew"], b["vw"]))


def sort_rows(rp, col, ew):
    col, ew = col.copy(), ew.copy()
    for x in range(rp.shape[0] - 1):
        s, e = rp[x], rp[x + 1]
        o = np.argsort(col[s:e], kind="stable")
        col[s:e] = col[s:e][o]
        ew[s:e] = ew[s:e][o]
    return col, ew


def assert_same_graph(a, b):
    rp_a, col_a, ew_a, vw_a = a
    rp_b, col_b, ew_b, vw_b = b
    assert np.array_equal(rp_a, rp_b)
    assert np.array_equal(vw_a, vw_b)
    ca, wa = sort_rows(rp_a, col_a, ew_a)
    cb, wb = sort_rows(rp_b, col_b, ew_b)
    assert np.array_equal(ca, cb) and np.array_equal(wa, wb)


def check_full(g, opts=None, trace=True):
    labels, res, gev = gpu_cluster(g, opts, trace=trace)
    ref, ores, oev = oracle.louvain_plus(g, oracle_params(opts), trace=trace, trace_passes=trace)
    if trace:
        compare_traces(gev, oev)
    assert np.array_equal(labels, ref)
    assert res["phi"] == ores["phi"]
    assert res["n_clusters"] == ores["n_clusters"]
    assert res["levels"] == ores["levels"]
    assert res["passes_total"] == ores["passes_total"]
    assert res["objective"] == ores["objective"]
    assert res["modularity"] == ores["modularity"]
    return res


# ------------------------------------------------------------------ tiny

def tiny_graph(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 70))
    p = float(rng.uniform(0.02, 0.5))
    rp, col, ew = gg.random_graph(n, p, seed, wmax=int(rng.integers(1, 9)))
    kind = seed % 4
    if kind == 0:
        return gg.modularity_inputs(rp, col, ew)
    if kind == 1:
        return gg.cpm_inputs(rp, col, ew, 1, int(rng.integers(2, 30)))
    vw = rng.integers(1, 6, size=n).astype(np.int64)
    lam = [(0, 1), (1, 1), (int(rng.integers(1, 5)), int(rng.integers(5, 40)))][seed % 3]
    return gg.Graph(rp, col, ew, vw, lam[0], lam[1])


@pytest.mark.parametrize("seed", range(40))
def test_tiny_random_graphs_every_pass(seed):
    check_full(tiny_graph(seed))


def test_tiny_louvain_without_uncoarsening():
    for seed in range(8):
        check_full(tiny_graph(seed), lc.Options(uncoarsen=False))


def test_tiny_other_schedules():
    opts = lc.Options(pass_limit=9, phi=[(1, 1), (0, 1), (1, 2)] * 3, eps=(3, 7), seed=12345)
    for seed in range(6):
        check_full(tiny_graph(100 + seed), opts)


# ---------------------------------------------------------- edge cases

def graph_from_edges(n, edges, obj="mod", lam=(1, 4), wmax=1, seed=0):
    src = [e[0] for e in edges]
    dst = [e[1] for e in edges]
    rp, col, ew = gg.from_edges(n, src, dst, seed=seed, wmin=1, wmax=wmax)
    if obj == "mod":
        g = gg.modularity_inputs(rp, col, ew)
        if g.lam_den == 0:
            g.lam_den = 1
        g.vw = np.maximum(g.vw, 1)
        return g
    return gg.cpm_inputs(rp, col, ew, *lam)


def test_edgeless_and_single_vertex():
    for n in (1, 2, 7):
        g = graph_from_edges(n, [], obj="cpm")
        labels, res, _ = gpu_cluster(g)
        assert np.array_equal(labels, np.arange(n))
        assert res["phi"] == 0 and res["n_clusters"] == n


def test_empty_graph():
    rp = np.zeros(1, np.int64)
    labels, res = lc.lc_cluster(dev(rp), dev(np.zeros(0, np.int32)), dev(np.zeros(0, np.int32)),
                                dev(np.zeros(0, np.int64)), 1, 2)
    assert labels.numel() == 0 and res["n_clusters"] == 0


def test_single_edge_and_path():
    check_full(graph_from_edges(2, [(0, 1)], obj="cpm", lam=(1, 3)))
    check_full(graph_from_edges(5, [(0, 1), (1, 2), (2, 3), (3, 4)], obj="cpm", lam=(1, 3)))


def test_star_hub_in_global_table_bin():
    """A hub of degree 9000 (> 4096) takes the global-memory table bin."""
    n = 9001
    edges = [(0, i) for i in range(1, n)] + [(i, i + 1) for i in range(1, n - 1, 2)]
    check_full(graph_from_edges(n, edges, wmax=5, seed=3), trace=False)
    check_full(graph_from_edges(n, edges, obj="cpm", lam=(1, 50), wmax=5, seed=3), trace=False)


def test_cliques_and_components():
    edges, off = [], 0
    for s in (3, 40, 300, 5):
        edges += [(off + a, off + b) for a in range(s) for b in range(a + 1, s)]
        off += s
    check_full(graph_from_edges(off, edges, obj="cpm", lam=(1, 2)), trace=False)
    check_full(graph_from_edges(off, edges), trace=False)


def test_lambda_extremes():
    rp, col, ew = gg.random_graph(60, 0.1, 7, wmax=4)
    for lam in ((0, 1), (1, 1), (1, 1000000)):
        check_full(gg.Graph(rp, col, ew, np.ones(60, np.int64), *lam))


# -------------------------------------------------------- workloads

def test_sbm_planted_10k_bitexact():
    """The planted-partition SBM workload: 10,000 vertices, 100 blocks."""
    res = check_full(gg.sbm_planted())
    assert res["modularity"] > 0.48


def degree_classes_graph(seed=0, lam=None):
    """Centres with degrees in every bin (20 .. 6000) over shared leaves, plus
    random leaf-leaf edges, so every kernel variant and the hub path run."""
    rng = np.random.default_rng(seed)
    n_leaves = 7000
    centres = [20, 100, 200, 400, 800, 1600, 3000, 6000]
    n = n_leaves + len(centres)
    src, dst = [], []
    for i, d in enumerate(centres):
        leaves = rng.choice(n_leaves, size=d, replace=False)
        src += [n_leaves + i] * d
        dst += leaves.tolist()
    extra = rng.integers(0, n_leaves, size=(20000, 2))
    src += extra[:, 0].tolist()
    dst += extra[:, 1].tolist()
    rp, col, ew = gg.from_edges(n, src, dst, seed=seed, wmin=1, wmax=6)
    if lam is None:
        return gg.modularity_inputs(rp, col, ew)
    return gg.cpm_inputs(rp, col, ew, *lam)


def test_every_degree_bin():
    check_full(degree_classes_graph(0), trace=True)
    check_full(degree_classes_graph(1, lam=(1, 40)), trace=False)


@pytest.mark.parametrize("scale", [12, 15, 16])
def test_rmat_bitexact(scale):
    """R-MAT with the Graph500 quadrants, weights in [1, 8], modularity.
    Scale 15 has hubs above 4096 (global-table bin) and many isolated vertices."""
    g = gg.rmat(scale)
    check_full(g, trace=(scale == 12))


def test_grid_cpm_bitexact():
    """3-D 7-point lattice 24^3 with 1% rewiring, CPM lambda = 1/100."""
    check_full(gg.grid_cpm(side=24), trace=True)


def test_sbm_small_batch_members():
    for (n, k, p_in, p_out, s) in gg.batched_sbm_params(6, seed=5, n_hi=3000):
        rp, col, ew = gg.sbm(n, k, p_in, p_out, s)
        check_full(gg.modularity_inputs(rp, col, ew), trace=False)


# ------------------------------------------------- step-level entry points

@pytest.mark.parametrize("seed", range(6))
def test_local_move_from_random_clustering(seed):
    g = gg.rmat(11, seed=seed + 20) if seed % 2 else gg.sbm_planted(n=1500, blocks=15, seed=seed)
    start = gg.random_labels(g.n, max(2, g.n // 10), seed)
    tr = lc.Trace()
    lab = dev(start)
    out, res = lc.lc_local_move(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num, g.lam_den,
                                lab, singleton_start=False, trace=tr)
    torch.cuda.synchronize()
    C_out, phi, oev = oracle.local_move(g, start, trace=True)
    assert np.array_equal(out.cpu().numpy(), C_out)
    assert res["phi"] == phi
    for e in oev:
        e["level"] = 0
        e["phase"] = "uncoarsen"
    compare_traces(tr.events, oev)


@pytest.mark.parametrize("seed", range(4))
def test_contract_random_dense_clustering(seed):
    g = gg.rmat(13, seed=seed + 40)
    lab = gg.random_labels(g.n, [1, 7, 500, g.n][seed], seed)
    _, lab = np.unique(lab, return_inverse=True)
    lab = lab.astype(np.int32)
    n_c = int(lab.max()) + 1
    rp, col, ew, vw = lc.lc_contract(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), dev(lab), n_c)
    torch.cuda.synchronize()
    ref = oracle.contract(g, lab, n_c)
    assert_same_graph((rp.cpu().numpy(), col.cpu().numpy(), ew.cpu().numpy(), vw.cpu().numpy()), ref)


@pytest.mark.parametrize("seed", range(4))
def test_objective_random_clustering(seed):
    g = tiny_graph(200 + seed) if seed < 2 else gg.rmat(12, seed=seed)
    lab = gg.random_labels(g.n, min(5, g.n), seed)
    res = lc.lc_objective(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num, g.lam_den, dev(lab))
    assert res["phi"] == oracle.objective(g, lab)
    assert res["n_clusters"] == len(np.unique(lab))


def test_host_buffer_entry_point_matches_device():
    g = gg.sbm_planted(n=3000, blocks=30, seed=9)
    a, ra, _ = gpu_cluster(g, trace=False)
    b, rb = lc.lc_cluster_host(g.row_ptr, g.col, g.ew, g.vw, g.lam_num, g.lam_den)
    assert np.array_equal(a, b) and ra["phi"] == rb["phi"]


def test_repeatable_across_calls():
    g = gg.rmat(14, seed=3)
    a, ra, _ = gpu_cluster(g, trace=False)
    b, rb, _ = gpu_cluster(g, lc.Options(profile=True), trace=False)
    assert np.array_equal(a, b) and ra["phi"] == rb["phi"]
    assert rb["kernel_ms"]["move"] > 0


# --------------------------------------------------------- validation

def test_validation_errors():
    base = graph_from_edges(6, [(0, 1), (1, 2), (2, 0), (3, 4), (4, 5)], obj="cpm")

    def run(rp, col, ew, vw, lam=(1, 4)):
        with pytest.raises(lc.LCError) as ei:
            lc.lc_cluster(dev(rp), dev(col), dev(ew), dev(vw), *lam)
        return ei.value.code

    rp, col, ew, vw = base.row_ptr, base.col, base.ew, base.vw
    ew2 = ew.copy()
    ew2[0] = 5  # asymmetric weight
    assert run(rp, col, ew2, vw) == 2
    col2 = col.copy()
    col2[0] = 0  # self-loop at vertex 0
    assert run(rp, col2, ew, vw) in (3, 4)
    ew3 = ew.copy()
    ew3[1] = 0
    assert run(rp, col, ew3, vw) == 5
    vw2 = vw.copy()
    vw2[2] = -1
    assert run(rp, col, ew, vw2) == 5
    assert run(rp, col, ew, vw, lam=(5, 4)) == 1
    big = vw.copy()
    big[:] = 1 << 40
    assert run(rp, col, ew, big, lam=(1, 1)) == 6


BIN_PLANS = [
    dict(),  # defaults
    dict(bins=(8, 16, 32, 128, 256, 256, 256, 256, 256)),  # every row above 256 is a hub
    dict(bins=(4, 16, 32, 64, 256, 512, 1024, 2048, 2048), hub_chunk=1024),  # no bin 8
    dict(bins=(8, 8, 8, 128, 128, 512, 512, 2048, 4096), hub_chunk=4096),  # empty lane bins
    dict(bins=(2, 3, 20, 100, 200, 300, 700, 1500, 3000), hub_chunk=256),
    dict(ab_threads=(0, 0, 128, 32, 32)),  # afterburner thread groups
    dict(ab_threads=(1, 16, 512, 512, 128), bins=(8, 16, 32, 128, 256, 512, 1024, 2048, 2048)),
    dict(ab_threads=(1, 16, 16, 32, 512)),  # half a warp per candidate in group 2
]


@pytest.mark.parametrize("plan", range(len(BIN_PLANS)))
def test_bin_plans_give_identical_results(plan):
    """The degree bins and hub chunks only decide which kernel handles a
    vertex (Section IV-C-2 leaves them open); every plan must give the
    oracle's labels, passes and objective."""
    for g in (gg.rmat(15, seed=3), gg.sbm_planted(n=4000, blocks=40, p_in=0.06, p_out=0.002, seed=4),
              gg.grid_cpm(side=16)):
        labels, res, ev = gpu_cluster(g, opts=lc.Options(**BIN_PLANS[plan]), trace=True)
        ref, ores, oev = oracle.louvain_plus(g, trace=True, trace_passes=True)
        assert np.array_equal(labels, ref), g.name
        assert res["phi"] == ores["phi"] and res["passes_total"] == ores["passes_total"], g.name
        compare_traces(ev, oev)


def test_invalid_bin_plans_rejected():
    g = gg.rmat(9, seed=1)
    for kw in (dict(bins=(8, 16, 32, 128, 256, 512, 1024, 2048, 5000)),  # above bin 8's capacity
               dict(bins=(8, 16, 32, 128, 100)),  # decreasing
               dict(hub_chunk=100), dict(hub_chunk=1 << 20),
               dict(ab_threads=(0, 0, 64)), dict(ab_threads=(32,)), dict(ab_threads=(0, 0, 0, 16)),
               dict(tables=1, bins=(8, 16, 32, 128, 256, 512, 1024, 2048, 2048))):
        with pytest.raises(lc.LCError) as e:
            gpu_cluster(g, opts=lc.Options(**kw))
        assert e.value.code == 1, kw  # LC_ERR_ARG


@pytest.mark.parametrize("plan", [0, 2])
def test_graph_replay_gives_identical_results(plan):
    """opts.graphs replays the repeated passes of each LocalMovePasses call
    from one captured CUDA graph (temperature read from the device): labels,
    objective and pass counts equal the oracle's, alone and in a batch."""
    graphs = [gg.rmat(14, seed=7), gg.sbm_planted(n=3000, blocks=30, p_in=0.05, p_out=0.002, seed=8),
              gg.grid_cpm(side=14), gg.rmat(8, seed=9)]
    opts = lc.Options(graphs=True, **BIN_PLANS[plan])
    for g in graphs:
        for uncoarsen in (True, False):
            o = lc.Options(graphs=True, uncoarsen=uncoarsen, **BIN_PLANS[plan])
            labels, res, _ = gpu_cluster(g, opts=o)
            ref, ores, _ = oracle.louvain_plus(g, oracle.Params(uncoarsen=uncoarsen))
            assert np.array_equal(labels, ref), (g.name, uncoarsen)
            assert res["phi"] == ores["phi"] and res["passes_total"] == ores["passes_total"], g.name
    pack = gg.pack(graphs)
    labels, res = lc.lc_cluster_batch(dev(pack["row_ptr"]), dev(pack["col"]), dev(pack["ew"]), dev(pack["vw"]),
                                      pack["graph_ptr"], pack["lam_num"], pack["lam_den"], opts=opts)
    labels = labels.cpu().numpy()
    gp = pack["graph_ptr"]
    for k, g in enumerate(graphs):
        ref, ores, _ = oracle.louvain_plus(g)
        assert np.array_equal(labels[gp[k]:gp[k + 1]], ref), g.name
        assert res[k]["phi"] == ores["phi"], g.name
    # on the legacy default stream too (the capture runs on a library stream)
    g = graphs[0]
    labels, res = lc.lc_cluster(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num, g.lam_den,
                                opts=opts, stream=torch.cuda.default_stream())
    torch.cuda.synchronize()
    assert np.array_equal(labels.cpu().numpy(), oracle.louvain_plus(g)[0])
