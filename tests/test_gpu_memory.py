"""Device memory at the boundary: scratch comes from the caller's provider
(PyTorch's caching allocator through the binding) or the library's private
pool, is all returned before a call ends, and never changes the device's
default memory pool.  The footprint estimate bounds what calls really hold,
and the server admits by it without handing LC_ERR_OOM to its callers."""
import ctypes

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
CU_MEMPOOL_ATTR_RELEASE_THRESHOLD = 4  # CUmemPool_attribute in cuda.h


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def default_pool_threshold() -> int:
    """Release threshold of the device's default pool, read through the
    driver API (the pool torch's cudaMallocAsync backend would use)."""
    cu = ctypes.CDLL("libcuda.so.1")
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), ctypes.c_int(torch.cuda.current_device())) == 0
    val = ctypes.c_uint64()
    assert cu.cuMemPoolGetAttribute(pool, ctypes.c_int(CU_MEMPOOL_ATTR_RELEASE_THRESHOLD),
                                    ctypes.byref(val)) == 0
    return val.value


def graphs():
    return [gg.sbm_planted(n=3000, blocks=30, p_in=0.05, p_out=0.002, seed=1), gg.rmat(14, seed=2),
            gg.grid_cpm(side=20)]


@pytest.mark.parametrize("allocator", ["torch", "library"])
def test_scratch_is_returned_and_default_pool_untouched(allocator):
    before_thr = default_pool_threshold()
    for g in graphs():
        args = (dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num, g.lam_den)
        labels = torch.empty(g.n, dtype=torch.int32, device=DEV)
        torch.cuda.synchronize()
        base = torch.cuda.memory_allocated()
        torch.cuda.reset_peak_memory_stats()
        _, res = lc.lc_cluster(*args, opts=lc.Options(allocator=allocator), labels_out=labels)
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base  # every scratch block given back
        grew = torch.cuda.max_memory_allocated() - base
        assert res["scratch_peak_bytes"] > 0
        if allocator == "torch":
            assert grew >= res["scratch_peak_bytes"]  # the scratch came from torch's allocator
        else:
            assert grew == 0  # torch's allocator was not used at all
        ref, ores, _ = oracle.louvain_plus(g)
        assert np.array_equal(labels.cpu().numpy(), ref) and res["phi"] == ores["phi"]
    lc.lc_release_memory()
    assert default_pool_threshold() == before_thr


def test_measured_peak_within_the_estimate():
    for g in graphs() + [gg.rmat(16, seed=1)]:
        _, res = lc.lc_cluster(dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw), g.lam_num, g.lam_den)
        est = lc.lc_scratch_estimate(g.n, g.nnz)
        assert 0 < res["scratch_peak_bytes"] <= est, (g.name, res["scratch_peak_bytes"], est)
    pack = gg.pack([gg.sbm_planted(n=500 + 100 * k, blocks=5, p_in=0.1, p_out=0.004, seed=k)
                    for k in range(8)])
    _, res = lc.lc_cluster_batch(dev(pack["row_ptr"]), dev(pack["col"]), dev(pack["ew"]), dev(pack["vw"]),
                                 pack["graph_ptr"], pack["lam_num"], pack["lam_den"])
    n, nnz = int(pack["row_ptr"].shape[0] - 1), int(pack["col"].shape[0])
    assert 0 < res[0]["scratch_peak_bytes"] <= lc.lc_scratch_estimate(n, nnz, count=8)


def test_provider_failure_gives_oom_and_returns_everything():
    """A provider that runs dry part-way: LC_ERR_OOM, every block it handed
    out comes back, and the next call is exact."""
    g = gg.rmat(13, seed=3)
    lib = lc.load()
    d = [dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw)]
    labels = torch.empty(g.n, dtype=torch.int32, device=DEV)
    csr = lc._Csr(g.n, g.nnz, d[0].data_ptr(), d[1].data_ptr())
    ref, ores, _ = oracle.louvain_plus(g)
    for budget in (0, 3, 17, 40):
        taken, live = [0], {}

        def alloc(ctx, nbytes, stream):
            if taken[0] >= budget:
                return None
            taken[0] += 1
            p = torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
            live[p] = nbytes
            return p

        def free(ctx, ptr, nbytes, stream):
            assert live.pop(int(ptr)) == nbytes
            torch.cuda.caching_allocator_delete(int(ptr))

        fa, ff = lc._AllocFn(alloc), lc._FreeFn(free)
        c = lc._c_opts(lc.Options(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        c.alloc, c.dealloc = fa, ff
        res = lc._Result()
        torch.cuda.synchronize()
        base = torch.cuda.memory_allocated()
        rc = lib.lc_cluster(ctypes.byref(csr), ctypes.c_void_p(d[3].data_ptr()),
                            ctypes.c_void_p(d[2].data_ptr()), g.lam_num, g.lam_den, ctypes.byref(c),
                            ctypes.c_void_p(labels.data_ptr()), ctypes.byref(res))
        torch.cuda.synchronize()
        assert rc == 7, (budget, rc)  # LC_ERR_OOM
        assert not live and torch.cuda.memory_allocated() == base
    out, res = lc.lc_cluster(*d, g.lam_num, g.lam_den)
    assert np.array_equal(out.cpu().numpy(), ref) and res["phi"] == ores["phi"]


def test_half_set_provider_is_rejected():
    g = gg.rmat(8, seed=1)
    lib = lc.load()
    d = [dev(g.row_ptr), dev(g.col), dev(g.ew), dev(g.vw)]
    labels = torch.empty(g.n, dtype=torch.int32, device=DEV)
    csr = lc._Csr(g.n, g.nnz, d[0].data_ptr(), d[1].data_ptr())
    c = lc._c_opts(lc.Options(allocator="library"), None)
    c.alloc = lc._TORCH_ALLOC  # no dealloc
    res = lc._Result()
    rc = lib.lc_cluster(ctypes.byref(csr), ctypes.c_void_p(d[3].data_ptr()), ctypes.c_void_p(d[2].data_ptr()),
                        g.lam_num, g.lam_den, ctypes.byref(c), ctypes.c_void_p(labels.data_ptr()),
                        ctypes.byref(res))
    assert rc == 1  # LC_ERR_ARG


def test_server_budget_just_above_one_job_never_reports_oom():
    """A budget just above the largest job's footprint, several slots: jobs
    mostly run one or two at a time, each under its reserved scratch limit,
    and none reports LC_ERR_OOM; every result equals the oracle's."""
    jobs = [gg.rmat(12, seed=k) for k in range(3)] + \
           [gg.sbm_planted(n=1500 + 300 * k, blocks=10, p_in=0.05, p_out=0.003, seed=k) for k in range(4)] + \
           [gg.grid_cpm(side=14)]
    fp = max(lc.lc_scratch_estimate(g.n, g.nnz) + 24 * (g.n + 1) + 8 * g.nnz + 5 * 512 for g in jobs)
    with lc.Server(slots=4, max_batch=4, hbm_budget=fp + fp // 8) as srv:
        ids = [srv.submit(g.row_ptr, g.col, g.ew, g.vw, g.lam_num, g.lam_den) for g in jobs]
        out = [srv.wait(j) for j in ids]  # raises LCError on any failure, OOM included
    for g, (labels, res, _) in zip(jobs, out):
        ref, ores, _ = oracle.louvain_plus(g)
        assert np.array_equal(labels, ref) and res["phi"] == ores["phi"]


def test_server_with_torch_provider_from_its_threads():
    jobs = [gg.rmat(10, seed=k) for k in range(6)]
    with lc.Server(slots=3, max_batch=2, opts=lc.Options(allocator="torch")) as srv:
        ids = [srv.submit(g.row_ptr, g.col, g.ew, g.vw, g.lam_num, g.lam_den) for g in jobs]
        out = [srv.wait(j) for j in ids]
    for g, (labels, res, _) in zip(jobs, out):
        ref, ores, _ = oracle.louvain_plus(g)
        assert np.array_equal(labels, ref) and res["phi"] == ores["phi"]
