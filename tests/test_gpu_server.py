"""Served form: requests submitted while others are running are admitted as
slots and memory free up, and every job's result equals the graph clustered
alone (and the oracle)."""
import random
import threading
import time

import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2608_01503_gb300 as lc  # noqa: E402


def request_graphs(seed=0, count=24):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        if k % 3 == 0:
            out.append(gg.rmat(int(rng.integers(8, 13)), seed=k))
        elif k % 3 == 1:
            out.append(gg.sbm_planted(n=int(rng.integers(300, 3000)), blocks=int(rng.integers(3, 30)),
                                      p_in=0.08, p_out=0.004, seed=k))
        else:
            rp, col, ew = gg.sbm(int(rng.integers(200, 2000)), 8, 0.06, 0.003, k, 1, 8)
            out.append(gg.cpm_inputs(rp, col, ew, 1, 50))
    return out


@pytest.mark.parametrize("slots,budget", [(3, 0), (2, 4 << 20)])
def test_served_results_equal_standalone(slots, budget):
    graphs = request_graphs(seed=slots)
    ids = [None] * len(graphs)
    with lc.Server(slots=slots, max_batch=5, hbm_budget=budget) as srv:
        def producer():
            rnd = random.Random(7)
            for k, g in enumerate(graphs):
                ids[k] = srv.submit(g.row_ptr, g.col, g.ew, g.vw, g.lam_num, g.lam_den)
                time.sleep(rnd.uniform(0, 0.004))

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        results = [srv.wait(j) for j in ids]
    for k, g in enumerate(graphs):
        labels, res, lat = results[k]
        ref, ores, _ = oracle.louvain_plus(g)
        assert np.array_equal(labels, ref), k
        assert res["phi"] == ores["phi"] and res["modularity"] == ores["modularity"], k
        assert lat >= 0


def test_poll_reports_not_ready_then_result():
    g = gg.rmat(12, seed=3)
    with lc.Server(slots=1) as srv:
        j = srv.submit(g.row_ptr, g.col, g.ew, g.vw, g.lam_num, g.lam_den)
        got = None
        for _ in range(20000):
            got = srv.poll(j)
            if got is not None:
                break
            time.sleep(0.001)
    assert got is not None
    ref, ores, _ = oracle.louvain_plus(g)
    assert np.array_equal(got[0], ref) and got[1]["phi"] == ores["phi"]


def test_bad_request_fails_alone():
    """An asymmetric graph and one over the exactness guard, admitted with
    good requests, fail with their own errors; the others equal the oracle."""
    good = [gg.rmat(10, seed=k) for k in range(3)]
    asym = gg.rmat(9, seed=9)
    ew_bad = asym.ew.copy()
    ew_bad[0] += 1  # (u,v) and (v,u) now differ
    heavy = gg.rmat(9, seed=8)
    ew_heavy = np.full_like(heavy.ew, 2**30)  # sum of edge weights beyond 2^31
    with lc.Server(slots=1, max_batch=16) as srv:
        ids = [srv.submit(g.row_ptr, g.col, g.ew, g.vw, g.lam_num, g.lam_den) for g in good[:2]]
        bad1 = srv.submit(asym.row_ptr, asym.col, ew_bad, asym.vw, asym.lam_num, asym.lam_den)
        bad2 = srv.submit(heavy.row_ptr, heavy.col, ew_heavy, heavy.vw, 1, 10**12)
        ids.append(srv.submit(good[2].row_ptr, good[2].col, good[2].ew, good[2].vw, good[2].lam_num,
                              good[2].lam_den))
        with pytest.raises(lc.LCError) as e1:
            srv.wait(bad1)
        with pytest.raises(lc.LCError) as e2:
            srv.wait(bad2)
        outs = [srv.wait(j) for j in ids]
    assert e1.value.code == 2 and e2.value.code == 6  # asymmetric, overflow
    for g, (labels, res, _) in zip(good, outs):
        ref, ores, _ = oracle.louvain_plus(g)
        assert np.array_equal(labels, ref) and res["phi"] == ores["phi"]


def test_cancel_a_queued_request():
    """With a 1-byte budget jobs run one at a time, so requests submitted
    while a large one runs stay queued and can be withdrawn."""
    big = gg.rmat(17, seed=1)
    small = [gg.rmat(9, seed=k) for k in range(3)]
    with lc.Server(slots=1, hbm_budget=1) as srv:
        jb = srv.submit(big.row_ptr, big.col, big.ew, big.vw, big.lam_num, big.lam_den)
        js = [srv.submit(g.row_ptr, g.col, g.ew, g.vw, g.lam_num, g.lam_den) for g in small]
        assert srv.cancel(js[1]) is True
        with pytest.raises(lc.LCError):
            lc.lc_server_wait(srv._h, js[1], 10)  # the id is gone
        out = {j: srv.wait(j) for j in (jb, js[0], js[2])}
    for g, j in ((big, jb), (small[0], js[0]), (small[2], js[2])):
        ref, ores, _ = oracle.louvain_plus(g)
        assert np.array_equal(out[j][0], ref) and out[j][1]["phi"] == ores["phi"]


def test_scratch_limit_gives_oom_and_leaves_no_state():
    g = gg.rmat(14, seed=2)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    args = (t(g.row_ptr), t(g.col), t(g.ew), t(g.vw), g.lam_num, g.lam_den)
    with pytest.raises(lc.LCError) as e:
        lc.lc_cluster(*args, opts=lc.Options(scratch_limit=1 << 20))
    assert e.value.code == 7  # LC_ERR_OOM
    ref, ores, _ = oracle.louvain_plus(g)
    for limit in (0, 8 << 30):
        labels, res = lc.lc_cluster(*args, opts=lc.Options(scratch_limit=limit))
        torch.cuda.synchronize()
        assert np.array_equal(labels.cpu().numpy(), ref) and res["phi"] == ores["phi"]


@pytest.mark.slow
def test_small_request_finishes_during_a_long_job():
    """A small request submitted while an R-MAT scale-21 job runs in another
    slot is done before that job is; both equal their standalone results."""
    big = gg.rmat(21, seed=11)
    small = gg.sbm_planted(n=1500, blocks=15, p_in=0.08, p_out=0.003, seed=4)
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    big_ref, big_res = lc.lc_cluster(t(big.row_ptr), t(big.col), t(big.ew), t(big.vw), big.lam_num, big.lam_den,
                                     opts=lc.Options(allocator="library"))
    big_ref = big_ref.cpu().numpy()
    with lc.Server(slots=2, max_batch=8) as srv:
        jb = srv.submit(big.row_ptr, big.col, big.ew, big.vw, big.lam_num, big.lam_den)
        time.sleep(0.005)  # the long job is admitted to the first slot
        js = srv.submit(small.row_ptr, small.col, small.ew, small.vw, small.lam_num, small.lam_den)
        s_labels, s_res, s_lat = srv.wait(js)
        assert srv.poll(jb) is None, "the long job finished before the small request"
        b_labels, b_res, b_lat = srv.wait(jb)
    assert s_lat < b_lat
    ref, ores, _ = oracle.louvain_plus(small)
    assert np.array_equal(s_labels, ref) and s_res["phi"] == ores["phi"]
    assert np.array_equal(b_labels, big_ref) and b_res["phi"] == big_res["phi"]
