"""Python binding of liblc — GB300 (sm_103a) pLouvain / Louvain+ on LambdaCC.

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``liblc.so`` behind the C ABI declared in ``include/lc.h``.  PyTorch
provides device memory (its caching allocator is passed to the library as
the scratch provider, ``Options.allocator = "torch"``, the default) and the
current CUDA stream.  If the native library is missing or cannot be loaded,
every call raises; there is no CPU path.

Functions carry the C names:
  lc_cluster        Louvain+ (Algorithm 1) on device tensors
  lc_cluster_batch  many graphs packed in one CSR, one launch per step for all
  lc_cluster_host   the same on host (numpy) buffers, copies included
  lc_cluster_constrained  Louvain+ with a constraint clustering (Section V-B)
  lc_cluster_iterated     iterated Louvain+ (each run constrained by the last)
  lc_cluster_leiden       pLeiden / pLeiden+ (Section V)
  lc_local_move     one LocalMovePasses call (Algorithm 2 + Algorithm 3)
  lc_contract       graph contraction (Algorithm 4)
  lc_objective      exact LambdaCC objective (Eq. 1)
  lc_objective_static  the same without allocating device memory
  lc_server_*       the clustering service: submit host graphs, poll/wait
                    for results; Server wraps it as a context manager
  lc_scratch_estimate  device scratch a call is expected to need
  lc_autotune       degree-bin boundaries, hub chunks and graph replay timed
                    on a workload (cached in tuning.json by load/save_tuning)
  lc_release_memory    return the library pool's cached blocks to the device
  lc_strerror       name of an error code
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from . import _build

_lib = None

LC_ERR_NOT_READY = 11

LC_K_NAMES = ["first_pass", "move", "afterburner", "apply", "objective", "contract", "other",
              "leiden_alt", "leiden_refine", "table"]


class LCError(RuntimeError):
    def __init__(self, code: int, detail: int = 0):
        self.code = code
        self.detail = detail
        super().__init__(f"liblc error {code}: {lc_strerror(code)} (detail {detail})")


class _Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p)]


class _Event(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("level", ctypes.c_int32), ("phase", ctypes.c_int32),
                ("pass_", ctypes.c_int32), ("n", ctypes.c_int64),
                ("labels", ctypes.POINTER(ctypes.c_int32)), ("dest", ctypes.POINTER(ctypes.c_int32)),
                ("moved", ctypes.POINTER(ctypes.c_uint8)),
                ("phi", ctypes.c_int64), ("count_L", ctypes.c_int64), ("count_M", ctypes.c_int64),
                ("cn", ctypes.c_int64), ("cnnz", ctypes.c_int64),
                ("c_row_ptr", ctypes.POINTER(ctypes.c_int64)), ("c_col", ctypes.POINTER(ctypes.c_int32)),
                ("c_ew", ctypes.POINTER(ctypes.c_int32)), ("c_vw", ctypes.POINTER(ctypes.c_int64))]


_EventFn = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.POINTER(_Event))
_AllocFn = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FreeFn = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


def _torch_alloc(_ctx, nbytes, stream):
    """lc_alloc_fn over PyTorch's caching allocator, on the call's stream."""
    import torch

    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
    except RuntimeError:  # out of memory: the call returns LC_ERR_OOM
        return None


def _torch_free(_ctx, ptr, _nbytes, _stream):
    import torch

    torch.cuda.caching_allocator_delete(int(ptr))


# module-level, so the C function pointers outlive every call
_TORCH_ALLOC = _AllocFn(_torch_alloc)
_TORCH_FREE = _FreeFn(_torch_free)


class _Opts(ctypes.Structure):
    _fields_ = [("pass_limit", ctypes.c_int32), ("phi_num", ctypes.c_int32 * 16),
                ("phi_den", ctypes.c_int32 * 16), ("eps_num", ctypes.c_int32),
                ("eps_den", ctypes.c_int32), ("seed", ctypes.c_uint32),
                ("uncoarsen", ctypes.c_int32), ("validate", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("event_cb", _EventFn), ("event_ctx", ctypes.c_void_p),
                ("symmetry", ctypes.c_int32), ("tables", ctypes.c_int32),
                ("scratch_limit", ctypes.c_int64), ("alloc", _AllocFn), ("dealloc", _FreeFn),
                ("alloc_ctx", ctypes.c_void_p), ("bin_max_deg", ctypes.c_int32 * 9),
                ("hub_chunk", ctypes.c_int32), ("ab_threads", ctypes.c_int32 * 5),
                ("graphs", ctypes.c_int32)]


class _Result(ctypes.Structure):
    _fields_ = [("n_clusters", ctypes.c_int64), ("levels", ctypes.c_int32),
                ("passes_total", ctypes.c_int32), ("phi", ctypes.c_int64),
                ("lambda_den", ctypes.c_int64), ("objective", ctypes.c_double),
                ("modularity", ctypes.c_double), ("edges_local_move", ctypes.c_int64),
                ("edges_contract", ctypes.c_int64), ("kernel_ms", ctypes.c_double * 10),
                ("kernel_launches", ctypes.c_int64 * 10), ("kernel_bytes", ctypes.c_double * 10),
                ("error_detail", ctypes.c_int64), ("tables_rebuilt", ctypes.c_int64),
                ("scratch_peak_bytes", ctypes.c_int64)]


class _Tuning(ctypes.Structure):
    _fields_ = [("bin_max_deg", ctypes.c_int32 * 9), ("hub_chunk", ctypes.c_int32),
                ("ab_threads", ctypes.c_int32 * 5), ("graphs", ctypes.c_int32), ("trials", ctypes.c_int32),
                ("ms_default", ctypes.c_double), ("ms_best", ctypes.c_double)]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("hbm_budget", ctypes.c_int64), ("opts", _Opts)]


EXPORTS = ["lc_default_opts", "lc_strerror", "lc_cluster", "lc_cluster_batch", "lc_cluster_host",
           "lc_local_move",
           "lc_cluster_constrained", "lc_cluster_iterated", "lc_cluster_leiden",
           "lc_contract", "lc_objective", "lc_objective_static", "lc_objective_static_max_vertices",
           "lc_server_default_config", "lc_server_create", "lc_server_submit", "lc_server_poll",
           "lc_server_wait", "lc_server_destroy", "lc_server_cancel", "lc_release_memory",
           "lc_scratch_estimate", "lc_autotune", "lc_debug_enabled", "lc_debug_selftest", "lc_check_opts"]


def library_path() -> str:
    """liblc.so, or the checked build liblc_debug.so when LC_DEBUG=1 is set."""
    return _build.lib_path()


def load(build_if_missing: bool = True):
    """Load liblc.so (building it in-tree if missing and allowed)."""
    global _lib
    if _lib is not None:
        return _lib
    debug = _build.debug_requested()
    path = _build.lib_path(debug)
    if not os.path.exists(path) or not _build.up_to_date(debug):
        if not build_if_missing:
            raise RuntimeError(f"{os.path.basename(path)} not built at {path}")
        _build.build(debug=debug)
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64, i32 = ctypes.c_int64, ctypes.c_int32
    csr, opts, res = ctypes.POINTER(_Csr), ctypes.POINTER(_Opts), ctypes.POINTER(_Result)
    lib.lc_default_opts.argtypes = [opts]
    lib.lc_default_opts.restype = None
    lib.lc_strerror.argtypes = [ctypes.c_int]
    lib.lc_strerror.restype = ctypes.c_char_p
    lib.lc_cluster.argtypes = [csr, P, P, i64, i64, opts, P, res]
    lib.lc_cluster_host.argtypes = [csr, P, P, i64, i64, opts, P, res]
    lib.lc_cluster_constrained.argtypes = [csr, P, P, i64, i64, P, opts, P, res]
    lib.lc_cluster_iterated.argtypes = [csr, P, P, i64, i64, i32, opts, P, res]
    lib.lc_cluster_leiden.argtypes = [csr, P, P, i64, i64, P, opts, P, res]
    lib.lc_cluster_batch.argtypes = [csr, P, P, i32, P, P, P, opts, P, res]
    lib.lc_local_move.argtypes = [csr, P, P, i64, i64, opts, P, i32, res]
    lib.lc_contract.argtypes = [csr, P, P, P, i64, opts, P, P, P, P, i64, ctypes.POINTER(i64)]
    lib.lc_objective.argtypes = [csr, P, P, i64, i64, P, opts, res]
    lib.lc_objective_static.argtypes = [csr, P, P, i64, i64, P, opts, res]
    lib.lc_objective_static_max_vertices.argtypes = []
    lib.lc_objective_static_max_vertices.restype = ctypes.c_int64
    lib.lc_release_memory.argtypes = []
    lib.lc_release_memory.restype = ctypes.c_int
    lib.lc_scratch_estimate.argtypes = [i64, i64, i32, opts]
    lib.lc_scratch_estimate.restype = ctypes.c_int64
    lib.lc_autotune.argtypes = [csr, P, P, i32, P, P, P, opts, i32, ctypes.POINTER(_Tuning)]
    lib.lc_autotune.restype = ctypes.c_int
    lib.lc_check_opts.argtypes = [opts]
    lib.lc_check_opts.restype = ctypes.c_int
    lib.lc_debug_enabled.argtypes = []
    lib.lc_debug_enabled.restype = ctypes.c_int
    lib.lc_debug_selftest.argtypes = [P, ctypes.POINTER(i64)]
    lib.lc_debug_selftest.restype = ctypes.c_int
    srv = ctypes.c_void_p
    lib.lc_server_default_config.argtypes = [ctypes.POINTER(_ServerConfig)]
    lib.lc_server_default_config.restype = None
    lib.lc_server_create.argtypes = [ctypes.POINTER(_ServerConfig), ctypes.POINTER(srv)]
    lib.lc_server_submit.argtypes = [srv, csr, P, P, i64, i64, ctypes.POINTER(i64)]
    lib.lc_server_poll.argtypes = [srv, i64, P, res, ctypes.POINTER(ctypes.c_double)]
    lib.lc_server_wait.argtypes = [srv, i64, P, res, ctypes.POINTER(ctypes.c_double)]
    lib.lc_server_destroy.argtypes = [srv]
    lib.lc_server_cancel.argtypes = [srv, i64]
    for f in ("lc_server_create", "lc_server_submit", "lc_server_poll", "lc_server_wait",
              "lc_server_destroy", "lc_server_cancel"):
        getattr(lib, f).restype = ctypes.c_int
    for f in ("lc_cluster", "lc_cluster_batch", "lc_cluster_host", "lc_local_move", "lc_contract",
              "lc_objective", "lc_objective_static"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def lc_strerror(code: int) -> str:
    return load().lc_strerror(code).decode()


@dataclass
class Options:
    """Mirror of lc_opts (defaults of Section VI-C)."""

    pass_limit: int = 6
    phi: list = field(default_factory=lambda: [(3, 4)] * 4 + [(1, 4)] * 2)
    eps: tuple = (1, 10)
    seed: int = 0
    uncoarsen: bool = True
    validate: bool = True
    profile: bool = False
    symmetry: int = 0  # 0 afterburner, 1 none, 2 minimum label heuristic in odd passes
    scratch_limit: int = 0  # bytes of device scratch a call may hold; 0 = no limit
    tables: int = 0  # 1: high-degree tables kept across passes and updated in place
    allocator: str = "torch"  # device scratch from PyTorch's caching allocator, or "library"
                              # for liblc's private pool
    bins: tuple = ()  # upper degrees of the 9 shared-memory bins (0 or missing = default)
    hub_chunk: int = 0  # edges per hub chunk (0 = default)
    graphs: bool = False  # replay the repeated passes of each LocalMovePasses call from a CUDA graph
    ab_threads: tuple = ()  # threads per candidate of the 5 afterburner groups (0 = default)


def _c_opts(o: Options | None, stream, event_fn=None) -> _Opts:
    o = o or Options()
    if o.allocator not in ("torch", "library"):
        raise ValueError(f"allocator must be 'torch' or 'library', not {o.allocator!r}")
    c = _Opts()
    load().lc_default_opts(ctypes.byref(c))
    c.pass_limit = o.pass_limit
    phi = list(o.phi) + [(1, 4)] * (16 - len(o.phi))
    for i in range(16):
        c.phi_num[i], c.phi_den[i] = phi[i]
    c.eps_num, c.eps_den = o.eps
    c.seed = o.seed & 0xFFFFFFFF
    c.uncoarsen = int(bool(o.uncoarsen))
    c.validate = int(bool(o.validate))
    c.profile = int(bool(o.profile))
    c.symmetry = int(o.symmetry)
    c.scratch_limit = int(o.scratch_limit)
    c.tables = int(o.tables)
    bins = list(o.bins) + [0] * (9 - len(o.bins))
    if len(bins) != 9:
        raise ValueError("bins holds at most 9 upper degrees")
    for k in range(9):
        c.bin_max_deg[k] = int(bins[k])
    c.hub_chunk = int(o.hub_chunk)
    abt = list(o.ab_threads) + [0] * (5 - len(o.ab_threads))
    if len(abt) != 5:
        raise ValueError("ab_threads holds at most 5 entries")
    for k in range(5):
        c.ab_threads[k] = int(abt[k])
    c.graphs = int(bool(o.graphs))
    c.stream = stream
    if event_fn is not None:
        c.event_cb = event_fn
    if o.allocator == "torch":
        c.alloc = _TORCH_ALLOC
        c.dealloc = _TORCH_FREE
    return c


def _stream_handle(stream=None):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, dtype, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr()) if t.numel() else ctypes.c_void_p(0)


def _result(r: _Result) -> dict:
    out = {k: getattr(r, k) for k in ("n_clusters", "levels", "passes_total", "phi", "lambda_den",
                                      "objective", "modularity", "edges_local_move", "edges_contract",
                                      "error_detail", "tables_rebuilt", "scratch_peak_bytes")}
    out["kernel_ms"] = dict(zip(LC_K_NAMES, list(r.kernel_ms)))
    out["kernel_launches"] = dict(zip(LC_K_NAMES, list(r.kernel_launches)))
    out["kernel_bytes"] = dict(zip(LC_K_NAMES, list(r.kernel_bytes)))
    return out


def _arr(ptr, n, dtype):
    if n == 0 or not ptr:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).copy()


class Trace:
    """Collects lc_event records (host copies) for parity checks."""

    def __init__(self):
        self.events = []
        self.fn = _EventFn(self._on)

    def _on(self, _ctx, evp):
        ev = evp.contents
        kind = {1: "pass", 2: "lmp", 3: "contract"}[ev.kind]
        rec = {"kind": kind, "level": ev.level, "phase": "coarsen" if ev.phase == 0 else "uncoarsen",
               "pass": ev.pass_, "n": ev.n, "C": _arr(ev.labels, ev.n, np.int32), "phi": ev.phi}
        if kind == "pass":
            rec.update(D=_arr(ev.dest, ev.n, np.int32), in_M=_arr(ev.moved, ev.n, np.uint8).astype(bool),
                       count_L=ev.count_L, count_M=ev.count_M)
        if kind == "contract":
            rec.update(cn=ev.cn, cnnz=ev.cnnz, row_ptr=_arr(ev.c_row_ptr, ev.cn + 1, np.int64),
                       col=_arr(ev.c_col, ev.cnnz, np.int32), ew=_arr(ev.c_ew, ev.cnnz, np.int32),
                       vw=_arr(ev.c_vw, ev.cn, np.int64))
        self.events.append(rec)


def _check(rc: int, res: _Result | None = None):
    if rc != 0:
        raise LCError(rc, res.error_detail if res is not None else 0)


def lc_cluster(row_ptr, col, ew, vw, lambda_num: int, lambda_den: int, opts: Options | None = None,
               labels_out=None, stream=None, trace: Trace | None = None):
    """Louvain+ on device tensors (row_ptr int64, col int32, ew int32, vw int64).
    Returns (labels int32 CUDA tensor, result dict)."""
    import torch

    lib = load()
    n = row_ptr.numel() - 1
    csr = _Csr(n, col.numel(), _dev(row_ptr, torch.int64, "row_ptr"), _dev(col, torch.int32, "col"))
    if labels_out is None:
        labels_out = torch.empty(max(n, 0), dtype=torch.int32, device=row_ptr.device)
    c = _c_opts(opts, _stream_handle(stream), trace.fn if trace else None)
    res = _Result()
    rc = lib.lc_cluster(ctypes.byref(csr), _dev(vw, torch.int64, "vw"), _dev(ew, torch.int32, "ew"),
                        int(lambda_num), int(lambda_den), ctypes.byref(c),
                        _dev(labels_out, torch.int32, "labels_out"), ctypes.byref(res))
    _check(rc, res)
    return labels_out, _result(res)


def lc_cluster_constrained(row_ptr, col, ew, vw, lambda_num: int, lambda_den: int, constraint,
                           opts: Options | None = None, labels_out=None, stream=None,
                           trace: Trace | None = None):
    """Louvain+ whose coarsening is constrained by `constraint` (int32 CUDA
    tensor, one label per vertex; Section V-B).  Returns (labels, result)."""
    import torch

    lib = load()
    n = row_ptr.numel() - 1
    if constraint.numel() != n:
        raise ValueError("constraint must have one label per vertex")
    csr = _Csr(n, col.numel(), _dev(row_ptr, torch.int64, "row_ptr"), _dev(col, torch.int32, "col"))
    if labels_out is None:
        labels_out = torch.empty(max(n, 0), dtype=torch.int32, device=row_ptr.device)
    c = _c_opts(opts, _stream_handle(stream), trace.fn if trace else None)
    res = _Result()
    rc = lib.lc_cluster_constrained(ctypes.byref(csr), _dev(vw, torch.int64, "vw"),
                                    _dev(ew, torch.int32, "ew"), int(lambda_num), int(lambda_den),
                                    _dev(constraint, torch.int32, "constraint"), ctypes.byref(c),
                                    _dev(labels_out, torch.int32, "labels_out"), ctypes.byref(res))
    _check(rc, res)
    return labels_out, _result(res)


def lc_cluster_iterated(row_ptr, col, ew, vw, lambda_num: int, lambda_den: int, iterations: int,
                        opts: Options | None = None, labels_out=None, stream=None):
    """Iterated Louvain+ (Section V-B): `iterations` runs, each after the
    first constrained by the previous output.  Returns (labels, result)."""
    import torch

    lib = load()
    n = row_ptr.numel() - 1
    csr = _Csr(n, col.numel(), _dev(row_ptr, torch.int64, "row_ptr"), _dev(col, torch.int32, "col"))
    if labels_out is None:
        labels_out = torch.empty(max(n, 0), dtype=torch.int32, device=row_ptr.device)
    c = _c_opts(opts, _stream_handle(stream))
    res = _Result()
    rc = lib.lc_cluster_iterated(ctypes.byref(csr), _dev(vw, torch.int64, "vw"),
                                 _dev(ew, torch.int32, "ew"), int(lambda_num), int(lambda_den),
                                 int(iterations), ctypes.byref(c),
                                 _dev(labels_out, torch.int32, "labels_out"), ctypes.byref(res))
    _check(rc, res)
    return labels_out, _result(res)


def lc_cluster_leiden(row_ptr, col, ew, vw, lambda_num: int, lambda_den: int, initial=None,
                      opts: Options | None = None, labels_out=None, stream=None,
                      trace: Trace | None = None):
    """pLeiden+ (opts.uncoarsen, the default) or pLeiden on device tensors;
    `initial`: optional int32 CUDA tensor of starting labels in [0, n).
    Returns (labels, result)."""
    import torch

    lib = load()
    n = row_ptr.numel() - 1
    csr = _Csr(n, col.numel(), _dev(row_ptr, torch.int64, "row_ptr"), _dev(col, torch.int32, "col"))
    if labels_out is None:
        labels_out = torch.empty(max(n, 0), dtype=torch.int32, device=row_ptr.device)
    c = _c_opts(opts, _stream_handle(stream), trace.fn if trace else None)
    res = _Result()
    init = ctypes.c_void_p(0) if initial is None else _dev(initial, torch.int32, "initial")
    rc = lib.lc_cluster_leiden(ctypes.byref(csr), _dev(vw, torch.int64, "vw"), _dev(ew, torch.int32, "ew"),
                               int(lambda_num), int(lambda_den), init, ctypes.byref(c),
                               _dev(labels_out, torch.int32, "labels_out"), ctypes.byref(res))
    _check(rc, res)
    return labels_out, _result(res)


def lc_cluster_batch(row_ptr, col, ew, vw, graph_ptr, lambda_num, lambda_den,
                     opts: Options | None = None, labels_out=None, stream=None):
    """Batched Louvain+ on a packed CSR (device tensors; graph_ptr, lambda_num
    and lambda_den are host sequences of length count+1, count, count).
    Returns (labels int32 CUDA tensor, numbered within each graph; list of
    per-graph result dicts)."""
    import torch

    lib = load()
    n = row_ptr.numel() - 1
    gp = np.ascontiguousarray(graph_ptr, dtype=np.int64)
    ln = np.ascontiguousarray(lambda_num, dtype=np.int64)
    ld = np.ascontiguousarray(lambda_den, dtype=np.int64)
    count = int(gp.shape[0] - 1)
    csr = _Csr(n, col.numel(), _dev(row_ptr, torch.int64, "row_ptr"), _dev(col, torch.int32, "col"))
    if labels_out is None:
        labels_out = torch.empty(max(n, 0), dtype=torch.int32, device=row_ptr.device)
    c = _c_opts(opts, _stream_handle(stream))
    res = (_Result * max(count, 1))()
    rc = lib.lc_cluster_batch(ctypes.byref(csr), _dev(vw, torch.int64, "vw"), _dev(ew, torch.int32, "ew"),
                              count, gp.ctypes.data, ln.ctypes.data, ld.ctypes.data, ctypes.byref(c),
                              _dev(labels_out, torch.int32, "labels_out"), res)
    _check(rc, res[0])
    return labels_out, [_result(res[k]) for k in range(count)]


def lc_cluster_host(row_ptr: np.ndarray, col: np.ndarray, ew: np.ndarray, vw: np.ndarray,
                    lambda_num: int, lambda_den: int, opts: Options | None = None,
                    labels_out: np.ndarray | None = None, stream=None):
    """Louvain+ on host arrays; the C call copies in and out itself."""
    lib = load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(ew, dtype=np.int32)
    v = np.ascontiguousarray(vw, dtype=np.int64)
    n = rp.shape[0] - 1
    if labels_out is None:
        labels_out = np.empty(max(n, 1), dtype=np.int32)
    csr = _Csr(n, cl.shape[0], rp.ctypes.data, cl.ctypes.data if cl.size else None)
    c = _c_opts(opts, _stream_handle(stream))
    res = _Result()
    rc = lib.lc_cluster_host(ctypes.byref(csr), v.ctypes.data if v.size else None,
                             w.ctypes.data if w.size else None, int(lambda_num), int(lambda_den),
                             ctypes.byref(c), labels_out.ctypes.data, ctypes.byref(res))
    _check(rc, res)
    return labels_out[:n], _result(res)


def lc_local_move(row_ptr, col, ew, vw, lambda_num: int, lambda_den: int, labels,
                  singleton_start: bool = False, opts: Options | None = None, stream=None,
                  trace: Trace | None = None):
    """One LocalMovePasses call; `labels` (int32 CUDA tensor) is replaced by C_out."""
    import torch

    lib = load()
    n = row_ptr.numel() - 1
    csr = _Csr(n, col.numel(), _dev(row_ptr, torch.int64, "row_ptr"), _dev(col, torch.int32, "col"))
    c = _c_opts(opts, _stream_handle(stream), trace.fn if trace else None)
    res = _Result()
    rc = lib.lc_local_move(ctypes.byref(csr), _dev(vw, torch.int64, "vw"), _dev(ew, torch.int32, "ew"),
                           int(lambda_num), int(lambda_den), ctypes.byref(c),
                           _dev(labels, torch.int32, "labels"), int(bool(singleton_start)),
                           ctypes.byref(res))
    _check(rc, res)
    return labels, _result(res)


def lc_contract(row_ptr, col, ew, vw, labels, n_c: int, opts: Options | None = None, stream=None):
    """Coarse graph of a dense clustering: (row_ptr, col, ew, vw) CUDA tensors."""
    import torch

    lib = load()
    n = row_ptr.numel() - 1
    dev = row_ptr.device
    csr = _Csr(n, col.numel(), _dev(row_ptr, torch.int64, "row_ptr"), _dev(col, torch.int32, "col"))
    cap = max(col.numel(), 1)
    c_rp = torch.empty(n_c + 1, dtype=torch.int64, device=dev)
    c_col = torch.empty(cap, dtype=torch.int32, device=dev)
    c_ew = torch.empty(cap, dtype=torch.int32, device=dev)
    c_vw = torch.empty(max(n_c, 1), dtype=torch.int64, device=dev)
    out_nnz = ctypes.c_int64(0)
    c = _c_opts(opts, _stream_handle(stream))
    rc = lib.lc_contract(ctypes.byref(csr), _dev(vw, torch.int64, "vw"), _dev(ew, torch.int32, "ew"),
                         _dev(labels, torch.int32, "labels"), int(n_c), ctypes.byref(c),
                         _dev(c_rp, torch.int64, "c_row_ptr"), _dev(c_col, torch.int32, "c_col"),
                         _dev(c_ew, torch.int32, "c_ew"), _dev(c_vw, torch.int64, "c_vw"), cap,
                         ctypes.byref(out_nnz))
    _check(rc)
    m = out_nnz.value
    return c_rp, c_col[:m], c_ew[:m], c_vw[:n_c]


def lc_objective(row_ptr, col, ew, vw, lambda_num: int, lambda_den: int, labels,
                 opts: Options | None = None, stream=None) -> dict:
    import torch

    lib = load()
    n = row_ptr.numel() - 1
    csr = _Csr(n, col.numel(), _dev(row_ptr, torch.int64, "row_ptr"), _dev(col, torch.int32, "col"))
    c = _c_opts(opts, _stream_handle(stream))
    res = _Result()
    rc = lib.lc_objective(ctypes.byref(csr), _dev(vw, torch.int64, "vw"), _dev(ew, torch.int32, "ew"),
                          int(lambda_num), int(lambda_den), _dev(labels, torch.int32, "labels"),
                          ctypes.byref(c), ctypes.byref(res))
    _check(rc, res)
    return _result(res)


def lc_scratch_estimate(n: int, nnz: int, count: int = 1, opts: Options | None = None) -> int:
    """Upper estimate of the device scratch lc_cluster (count = 1) or
    lc_cluster_batch needs for n vertices and nnz stored edges (bytes)."""
    c = _c_opts(opts, None)
    return int(load().lc_scratch_estimate(int(n), int(nnz), int(count), ctypes.byref(c)))


def lc_autotune(row_ptr, col, ew, vw, lambda_num, lambda_den, graph_ptr=None,
                opts: Options | None = None, repeats: int = 3, stream=None) -> dict:
    """Times the degree-bin boundaries, hub chunk length and graph replay on
    this workload (one graph, or a packed batch with host graph_ptr and
    per-graph lambda sequences) and returns the fastest setting, which gives
    identical results: {"bins", "hub_chunk", "graphs", "trials",
    "ms_default", "ms_best"}.  tuned_options() turns it into Options."""
    import torch

    lib = load()
    n = row_ptr.numel() - 1
    csr = _Csr(n, col.numel(), _dev(row_ptr, torch.int64, "row_ptr"), _dev(col, torch.int32, "col"))
    if graph_ptr is None:
        count, gp = 1, None
        ln = np.array([lambda_num], dtype=np.int64)
        ld = np.array([lambda_den], dtype=np.int64)
    else:
        gp = np.ascontiguousarray(graph_ptr, dtype=np.int64)
        ln = np.ascontiguousarray(lambda_num, dtype=np.int64)
        ld = np.ascontiguousarray(lambda_den, dtype=np.int64)
        count = int(gp.shape[0] - 1)
    c = _c_opts(opts, _stream_handle(stream))
    t = _Tuning()
    rc = lib.lc_autotune(ctypes.byref(csr), _dev(vw, torch.int64, "vw"), _dev(ew, torch.int32, "ew"), count,
                         gp.ctypes.data if gp is not None else None, ln.ctypes.data, ld.ctypes.data,
                         ctypes.byref(c), int(repeats), ctypes.byref(t))
    _check(rc)
    return {"bins": list(t.bin_max_deg), "hub_chunk": t.hub_chunk, "ab_threads": list(t.ab_threads),
            "graphs": bool(t.graphs),
            "trials": t.trials, "ms_default": t.ms_default, "ms_best": t.ms_best}


def tuned_options(tuning: dict | None, **kw) -> Options:
    """Options carrying a tuning (lc_autotune / load_tuning); None: defaults."""
    if tuning:
        kw.setdefault("bins", tuple(tuning["bins"]))
        kw.setdefault("hub_chunk", int(tuning["hub_chunk"]))
        kw.setdefault("ab_threads", tuple(tuning.get("ab_threads", ())))
        kw.setdefault("graphs", bool(tuning["graphs"]))
    return Options(**kw)


TUNING_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")


def load_tuning(key: str, path: str = TUNING_CACHE) -> dict | None:
    """A cached tuning for `key` (a workload and device name), or None."""
    import json

    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f).get(key)


def save_tuning(key: str, tuning: dict, path: str = TUNING_CACHE) -> None:
    import json

    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[key] = tuning
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
        f.write("\n")


def lc_release_memory() -> None:
    """Returns the blocks cached in liblc's private pool on the current device."""
    _check(load().lc_release_memory())


def lc_check_opts(opts: Options | None = None) -> None:
    """Raises LCError (LC_ERR_ARG) if the options are not a valid set for the
    clustering calls; host arithmetic only, no device needed."""
    c = _c_opts(opts, None)
    _check(load().lc_check_opts(ctypes.byref(c)))


def lc_debug_enabled() -> bool:
    """True when the loaded library is the checked build (LC_DEBUG=1)."""
    return bool(load().lc_debug_enabled())


def lc_debug_selftest(stream=None) -> int:
    """Checked build: one deliberate index-check failure, collected and
    decoded by the library; returns the encoded detail (site << 56 | index)."""
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    detail = ctypes.c_int64(0)
    _check(load().lc_debug_selftest(ctypes.c_void_p(s.cuda_stream), ctypes.byref(detail)), detail.value)
    return int(detail.value)


def lc_objective_static_max_vertices() -> int:
    return int(load().lc_objective_static_max_vertices())


def lc_objective_static(row_ptr, col, ew, vw, lambda_num: int, lambda_den: int, labels,
                        stream=None) -> dict:
    """lc_objective without any device allocation (for callers that cannot
    allocate at that point: a pool that owns the whole GPU, or a service
    that forbids cudaMalloc after start-up).  Scratch is a fixed array in
    the library; graphs above lc_objective_static_max_vertices() vertices
    are rejected.  Calls overlapping on the GPU race on that array."""
    import torch

    lib = load()
    n = row_ptr.numel() - 1
    csr = _Csr(n, col.numel(), _dev(row_ptr, torch.int64, "row_ptr"), _dev(col, torch.int32, "col"))
    c = _c_opts(Options(allocator="library"), _stream_handle(stream))  # it allocates nothing
    res = _Result()
    rc = lib.lc_objective_static(ctypes.byref(csr), _dev(vw, torch.int64, "vw"),
                                 _dev(ew, torch.int32, "ew"), int(lambda_num), int(lambda_den),
                                 _dev(labels, torch.int32, "labels"), ctypes.byref(c), ctypes.byref(res))
    _check(rc, res)
    return _result(res)



def lc_server_default_config() -> _ServerConfig:
    cfg = _ServerConfig()
    load().lc_server_default_config(ctypes.byref(cfg))
    return cfg


def lc_server_create(slots: int = 4, max_batch: int = 64, hbm_budget: int = 0,
                     opts: Options | None = None) -> ctypes.c_void_p:
    """Starts a clustering service on the current device; returns its handle."""
    cfg = lc_server_default_config()
    cfg.slots, cfg.max_batch, cfg.hbm_budget = slots, max_batch, hbm_budget
    # the slots' own threads allocate; the library's pool unless asked otherwise
    cfg.opts = _c_opts(opts or Options(allocator="library"), None)
    h = ctypes.c_void_p()
    _check(load().lc_server_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def lc_server_submit(server, row_ptr, col, ew, vw, lambda_num: int, lambda_den: int) -> int:
    """Queues one host graph (arrays are copied before return); returns the job id."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(ew, dtype=np.int32)
    v = np.ascontiguousarray(vw, dtype=np.int64)
    csr = _Csr(rp.shape[0] - 1, cl.shape[0], rp.ctypes.data, cl.ctypes.data if cl.size else None)
    jid = ctypes.c_int64()
    _check(load().lc_server_submit(server, ctypes.byref(csr), v.ctypes.data if v.size else None,
                                   w.ctypes.data if w.size else None, int(lambda_num),
                                   int(lambda_den), ctypes.byref(jid)))
    return jid.value


def _server_take(fn, server, jid: int, n: int):
    lab = np.empty(max(n, 1), dtype=np.int32)
    res = _Result()
    lat = ctypes.c_double()
    rc = fn(server, jid, lab.ctypes.data, ctypes.byref(res), ctypes.byref(lat))
    if rc == LC_ERR_NOT_READY:
        return None
    _check(rc, res)
    return lab[:n], _result(res), lat.value


def lc_server_poll(server, jid: int, n: int):
    """(labels, result, latency seconds) of a finished job, None while it runs."""
    return _server_take(load().lc_server_poll, server, jid, n)


def lc_server_wait(server, jid: int, n: int):
    """Blocks until the job is done; (labels, result, latency seconds)."""
    return _server_take(load().lc_server_wait, server, jid, n)


def lc_server_cancel(server, jid: int) -> bool:
    """Withdraws a queued job: True if it was withdrawn, False if it already
    runs or is done."""
    rc = load().lc_server_cancel(server, jid)
    if rc == LC_ERR_NOT_READY:
        return False
    _check(rc)
    return True


def lc_server_destroy(server) -> None:
    _check(load().lc_server_destroy(server))


class Server:
    """Context-manager wrapper of lc_server_*: requests are host graphs,
    admitted by device-memory footprint into `slots` concurrent batched runs."""

    def __init__(self, slots: int = 4, max_batch: int = 64, hbm_budget: int = 0,
                 opts: Options | None = None):
        self._h = lc_server_create(slots, max_batch, hbm_budget, opts)
        self._n = {}

    def submit(self, row_ptr, col, ew, vw, lambda_num: int, lambda_den: int) -> int:
        jid = lc_server_submit(self._h, row_ptr, col, ew, vw, lambda_num, lambda_den)
        self._n[jid] = len(row_ptr) - 1
        return jid

    def poll(self, jid: int):
        got = lc_server_poll(self._h, jid, self._n[jid])
        if got is not None:
            del self._n[jid]
        return got

    def wait(self, jid: int):
        got = lc_server_wait(self._h, jid, self._n[jid])
        del self._n[jid]
        return got

    def cancel(self, jid: int) -> bool:
        done = lc_server_cancel(self._h, jid)
        if done:
            del self._n[jid]
        return done

    def close(self):
        if self._h:
            lc_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
