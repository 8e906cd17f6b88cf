"""CPU oracle of pLouvain / Louvain+ on LambdaCC — TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never touches it, and the two share no code.

The arithmetic lives in ``lc_oracle.c`` (plain sequential C, int64/int128),
compiled in-tree with gcc on first use.  This file only marshals arguments.

Functions follow the paper's passages:
  objective     Eq. 1 (Phi = Lambda * lambdaCC, exact integer)
  gain          Section II-A: Lambda * w'(v, X)
  local_move    Algorithm 2 with Algorithm 3 (LocalMovePasses)
  contract      Section III-A coarse graph (the result Algorithm 4 computes)
  louvain_plus  Algorithm 1 (Louvain+; Louvain with uncoarsen=False)
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lc_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_LIB_OMP = os.path.join(_LIBDIR, "liboracle_omp.so")

GCC_FLAGS = ["-O2", "-std=gnu11", "-shared", "-fPIC", "-Wall", "-Wextra", "-Wno-unknown-pragmas"]

NONE = -1
EMPTY = -2


def build(force: bool = False, openmp: bool = False) -> str:
    """Compiles lc_oracle.c: sequentially, or with -fopenmp (the same source,
    its pass and contraction loops spread over the host's cores with
    identical results; the all-core CPU baseline)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    lib = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *GCC_FLAGS, *(["-fopenmp"] if openmp else []), _SRC, "-o", tmp])
        os.replace(tmp, lib)
    return lib


class _Graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("ew", ctypes.c_void_p), ("vw", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("lam_num", ctypes.c_int64), ("lam_den", ctypes.c_int64),
                ("pass_limit", ctypes.c_int32),
                ("phi_num", ctypes.c_int32 * 16), ("phi_den", ctypes.c_int32 * 16),
                ("eps_num", ctypes.c_int32), ("eps_den", ctypes.c_int32),
                ("seed", ctypes.c_uint32), ("uncoarsen", ctypes.c_int32), ("symmetry", ctypes.c_int32)]


class _Event(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("level", ctypes.c_int32), ("phase", ctypes.c_int32),
                ("pass_", ctypes.c_int32), ("n", ctypes.c_int64),
                ("C_before", ctypes.POINTER(ctypes.c_int32)), ("C", ctypes.POINTER(ctypes.c_int32)),
                ("D", ctypes.POINTER(ctypes.c_int32)),
                ("in_L", ctypes.POINTER(ctypes.c_uint8)), ("in_M", ctypes.POINTER(ctypes.c_uint8)),
                ("delta", ctypes.POINTER(ctypes.c_int64)), ("q", ctypes.POINTER(ctypes.c_int64)),
                ("adj", ctypes.POINTER(ctypes.c_int64)),
                ("phi_hi", ctypes.c_int64), ("phi_lo", ctypes.c_uint64),
                ("count_L", ctypes.c_int64), ("count_M", ctypes.c_int64),
                ("cn", ctypes.c_int64), ("cnnz", ctypes.c_int64),
                ("c_row_ptr", ctypes.POINTER(ctypes.c_int64)), ("c_col", ctypes.POINTER(ctypes.c_int32)),
                ("c_ew", ctypes.POINTER(ctypes.c_int32)), ("c_vw", ctypes.POINTER(ctypes.c_int64))]


class _Result(ctypes.Structure):
    _fields_ = [("n_clusters", ctypes.c_int64), ("levels", ctypes.c_int32),
                ("passes_total", ctypes.c_int32), ("phi_hi", ctypes.c_int64),
                ("phi_lo", ctypes.c_uint64), ("objective", ctypes.c_double),
                ("modularity", ctypes.c_double)]


_CB = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.POINTER(_Event))
_lib = None


def _bind(lib):
    """Declares the C signatures on a loaded build of lc_oracle.c."""
    G, P = ctypes.POINTER(_Graph), ctypes.POINTER(_Params)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.orc_objective.argtypes = [G, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, i64p,
                                  ctypes.POINTER(ctypes.c_uint64)]
    lib.orc_gain.argtypes = [G, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                             ctypes.c_int32, i64p]
    lib.orc_local_move.argtypes = [G, P, ctypes.c_void_p, _CB, ctypes.c_void_p, i64p,
                                   ctypes.POINTER(ctypes.c_uint64)]
    lib.orc_contract.argtypes = [G, ctypes.c_void_p, ctypes.c_int64, i64p, i64p,
                                 ctypes.POINTER(ctypes.POINTER(ctypes.c_int64)),
                                 ctypes.POINTER(ctypes.POINTER(ctypes.c_int32)),
                                 ctypes.POINTER(ctypes.POINTER(ctypes.c_int32)),
                                 ctypes.POINTER(ctypes.POINTER(ctypes.c_int64))]
    lib.orc_louvain_plus.argtypes = [G, P, ctypes.c_void_p, ctypes.POINTER(_Result), _CB,
                                     ctypes.c_void_p]
    lib.orc_louvain_plus_constrained.argtypes = [G, P, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.POINTER(_Result), _CB, ctypes.c_void_p]
    lib.orc_louvain_plus_iterated.argtypes = [G, P, ctypes.c_int32, ctypes.c_void_p,
                                              ctypes.POINTER(_Result), _CB, ctypes.c_void_p]
    lib.orc_pleiden.argtypes = [G, P, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(_Result), _CB,
                                ctypes.c_void_p]
    lib.orc_local_move_alt.argtypes = [G, P, ctypes.c_void_p, i64p]
    lib.orc_pleiden_refine.argtypes = [G, P, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    lib.orc_rand.argtypes = [ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64]
    lib.orc_rand.restype = ctypes.c_uint64
    lib.orc_free.argtypes = [ctypes.c_void_p]
    for f in (lib.orc_objective, lib.orc_gain, lib.orc_local_move, lib.orc_contract,
              lib.orc_louvain_plus, lib.orc_louvain_plus_constrained,
              lib.orc_louvain_plus_iterated, lib.orc_pleiden, lib.orc_local_move_alt,
              lib.orc_pleiden_refine):
        f.restype = ctypes.c_int
    return lib


_load_lock = threading.Lock()


def _load():
    global _lib
    with _load_lock:  # threads (louvain_plus_many) may arrive together
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


@contextlib.contextmanager
def all_cores():
    """Runs the oracle's OpenMP build while the context is open: the same
    passes and contractions, each loop over vertices or clusters spread over
    the host's cores (OMP_NUM_THREADS, else all of them)."""
    with library(build(openmp=True)):
        yield


@contextlib.contextmanager
def library(path: str):
    """Runs every oracle function against another build of lc_oracle.c while
    the context is open.  The tests compile copies with planted mistakes and
    check that the pins reject them."""
    global _lib
    saved = _lib
    _lib = _bind(ctypes.CDLL(os.path.abspath(path)))
    try:
        yield
    finally:
        _lib = saved


@dataclass
class Params:
    """Settings of the method (Section VI-C defaults: pass limit 6, phi 0.75
    for passes 1-4 and 0.25 for passes 5-6, epsilon 0.1)."""

    pass_limit: int = 6
    phi: list = field(default_factory=lambda: [(3, 4)] * 4 + [(1, 4)] * 2)
    eps: tuple = (1, 10)
    seed: int = 0
    uncoarsen: bool = True
    symmetry: int = 0  # 0 afterburner, 1 none, 2 minimum label heuristic in odd passes


def _c_params(lam_num: int, lam_den: int, p: Params) -> _Params:
    cp = _Params()
    cp.lam_num, cp.lam_den = int(lam_num), int(lam_den)
    cp.pass_limit = p.pass_limit
    phi = list(p.phi) + [(0, 1)] * (16 - len(p.phi))
    for i in range(16):
        cp.phi_num[i], cp.phi_den[i] = phi[i]
    cp.eps_num, cp.eps_den = p.eps
    cp.seed = p.seed & 0xFFFFFFFF
    cp.uncoarsen = 1 if p.uncoarsen else 0
    cp.symmetry = int(p.symmetry)
    return cp


class _Holder:
    """Keeps the numpy arrays alive while C holds their pointers."""

    def __init__(self, rp, col, ew, vw):
        self.rp = np.ascontiguousarray(rp, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.ew = np.ascontiguousarray(ew, dtype=np.int32)
        self.vw = np.ascontiguousarray(vw, dtype=np.int64)
        self.g = _Graph(self.rp.shape[0] - 1, self.col.shape[0], self.rp.ctypes.data,
                        self.col.ctypes.data if self.col.size else None,
                        self.ew.ctypes.data if self.ew.size else None,
                        self.vw.ctypes.data if self.vw.size else None)


def _graph(g):
    return _Holder(g.row_ptr, g.col, g.ew, g.vw)


def _i128(hi: int, lo: int) -> int:
    return (hi << 64) | lo


def _rc(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def objective(g, labels, lam_num=None, lam_den=None) -> int:
    """Phi(C) = Lambda * lambdaCC(C) (Eq. 1) as an exact Python int."""
    h = _graph(g)
    C = np.ascontiguousarray(labels, dtype=np.int32)
    hi, lo = ctypes.c_int64(), ctypes.c_uint64()
    mu = g.lam_num if lam_num is None else lam_num
    Lam = g.lam_den if lam_den is None else lam_den
    _rc(_load().orc_objective(ctypes.byref(h.g), mu, Lam, C.ctypes.data, ctypes.byref(hi),
                              ctypes.byref(lo)), "objective")
    return _i128(hi.value, lo.value)


def gain(g, labels, v: int, X: int) -> int:
    """g(v, X) = Lambda * w'(v, X); X = EMPTY for a new cluster."""
    h = _graph(g)
    C = np.ascontiguousarray(labels, dtype=np.int32)
    out = ctypes.c_int64()
    _rc(_load().orc_gain(ctypes.byref(h.g), g.lam_num, g.lam_den, C.ctypes.data, v, X,
                         ctypes.byref(out)), "gain")
    return out.value


def _arr(ptr, n, dtype):
    if n == 0 or not ptr:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).copy()


class _Recorder:
    def __init__(self, passes: bool):
        self.passes = passes
        self.events = []

    def __call__(self, _ctx, evp):
        ev = evp.contents
        n = ev.n
        rec = {"kind": {1: "pass", 2: "lmp", 3: "contract"}[ev.kind], "level": ev.level,
               "phase": "coarsen" if ev.phase == 0 else "uncoarsen", "pass": ev.pass_, "n": n}
        if ev.kind == 1:
            if not self.passes:
                return
            rec.update(C_before=_arr(ev.C_before, n, np.int32), C=_arr(ev.C, n, np.int32),
                       D=_arr(ev.D, n, np.int32), in_L=_arr(ev.in_L, n, np.uint8).astype(bool),
                       in_M=_arr(ev.in_M, n, np.uint8).astype(bool),
                       delta=_arr(ev.delta, n, np.int64), q=_arr(ev.q, n, np.int64),
                       adj=_arr(ev.adj, n, np.int64), phi=_i128(ev.phi_hi, ev.phi_lo),
                       count_L=ev.count_L, count_M=ev.count_M)
        elif ev.kind == 2:
            rec.update(C=_arr(ev.C, n, np.int32), phi=_i128(ev.phi_hi, ev.phi_lo))
        else:
            rec.update(C=_arr(ev.C, n, np.int32), cn=ev.cn, cnnz=ev.cnnz,
                       row_ptr=_arr(ev.c_row_ptr, ev.cn + 1, np.int64),
                       col=_arr(ev.c_col, ev.cnnz, np.int32), ew=_arr(ev.c_ew, ev.cnnz, np.int32),
                       vw=_arr(ev.c_vw, ev.cn, np.int64))
        self.events.append(rec)


def local_move(g, labels, params: Params | None = None, trace: bool = False):
    """One LocalMovePasses call (Algorithm 2) from `labels`.
    Returns (C_out, Phi(C_out), events)."""
    p = params or Params()
    h = _graph(g)
    C = np.ascontiguousarray(labels, dtype=np.int32).copy()
    cp = _c_params(g.lam_num, g.lam_den, p)
    rec = _Recorder(passes=trace)
    cb = _CB(rec)
    hi, lo = ctypes.c_int64(), ctypes.c_uint64()
    _rc(_load().orc_local_move(ctypes.byref(h.g), ctypes.byref(cp), C.ctypes.data, cb, None,
                               ctypes.byref(hi), ctypes.byref(lo)), "local_move")
    return C, _i128(hi.value, lo.value), rec.events


def contract(g, labels, n_c: int):
    """Coarse graph for a dense clustering in [0, n_c): (row_ptr, col, ew, vw)."""
    h = _graph(g)
    C = np.ascontiguousarray(labels, dtype=np.int32)
    on, onnz = ctypes.c_int64(), ctypes.c_int64()
    rp = ctypes.POINTER(ctypes.c_int64)()
    col = ctypes.POINTER(ctypes.c_int32)()
    ew = ctypes.POINTER(ctypes.c_int32)()
    vw = ctypes.POINTER(ctypes.c_int64)()
    lib = _load()
    _rc(lib.orc_contract(ctypes.byref(h.g), C.ctypes.data, n_c, ctypes.byref(on), ctypes.byref(onnz),
                         ctypes.byref(rp), ctypes.byref(col), ctypes.byref(ew), ctypes.byref(vw)),
        "contract")
    out = (_arr(rp, on.value + 1, np.int64), _arr(col, onnz.value, np.int32),
           _arr(ew, onnz.value, np.int32), _arr(vw, on.value, np.int64))
    for ptr in (rp, col, ew, vw):
        lib.orc_free(ctypes.cast(ptr, ctypes.c_void_p))
    return out


def louvain_plus(g, params: Params | None = None, trace: bool = False, trace_passes: bool = False):
    """Algorithm 1.  Returns (labels, result dict, events).  With trace=True the
    events hold every LocalMovePasses result and coarse graph; trace_passes
    adds every pass's intermediate state."""
    return _run(g, params, trace, trace_passes, "louvain_plus")


def louvain_plus_many(graphs, params: Params | None = None, threads: int | None = None):
    """louvain_plus on every graph (no trace), the graphs spread over host
    threads: the C calls release the GIL and share nothing, so each result
    is what one call alone returns.  Returns [(labels, result dict)]."""
    import concurrent.futures as cf

    def one(g):
        labels, res, _ = louvain_plus(g, params)
        return labels, res

    _load()
    # largest first, so the long runs do not start last
    order = sorted(range(len(graphs)), key=lambda k: -graphs[k].nnz)
    out = [None] * len(graphs)
    with cf.ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 4) as ex:
        for k, r in zip(order, ex.map(one, [graphs[k] for k in order])):
            out[k] = r
    return out


def louvain_plus_constrained(g, constraint, params: Params | None = None, trace: bool = False,
                             trace_passes: bool = False):
    """Algorithm 1 with its coarsening constrained by the clustering
    `constraint` (int32 >= 0 per vertex; Section V-B).  Same returns."""
    B = np.ascontiguousarray(constraint, dtype=np.int32)
    if B.shape[0] != g.n:
        raise ValueError("constraint must have one entry per vertex")
    return _run(g, params, trace, trace_passes, "louvain_plus_constrained", B)


def louvain_plus_iterated(g, iterations: int, params: Params | None = None, trace: bool = False,
                          trace_passes: bool = False):
    """Iterated Louvain+ (Section V-B): `iterations` runs in total, each after
    the first constrained by the previous output."""
    return _run(g, params, trace, trace_passes, "louvain_plus_iterated", iterations)


def pleiden(g, params: Params | None = None, C_in=None, trace: bool = False, trace_passes: bool = False):
    """pLeiden (Algorithm 5); with params.uncoarsen (the default) pLeiden+.
    C_in: initial clustering (labels in [0, n)), None for singletons."""
    C = None if C_in is None else np.ascontiguousarray(C_in, dtype=np.int32)
    return _run(g, params, trace, trace_passes, "pleiden", C)


def local_move_alt(g, labels, params: Params | None = None):
    """One LocalMoveAlt call (Section V-A).  Returns (C, moves committed)."""
    p = params or Params()
    h = _graph(g)
    C = np.ascontiguousarray(labels, dtype=np.int32).copy()
    k = ctypes.c_int64()
    _rc(_load().orc_local_move_alt(ctypes.byref(h.g), ctypes.byref(_c_params(g.lam_num, g.lam_den, p)),
                                   C.ctypes.data, ctypes.byref(k)), "local_move_alt")
    return C, k.value


def pleiden_refine(g, B, level: int = 0, params: Params | None = None):
    """One pLeidenR call (Algorithm 6) with constraint B; refined labels
    (root ids, not compacted)."""
    p = params or Params()
    h = _graph(g)
    Bc = np.ascontiguousarray(B, dtype=np.int32)
    R = np.zeros(max(g.n, 1), dtype=np.int32)
    _rc(_load().orc_pleiden_refine(ctypes.byref(h.g), ctypes.byref(_c_params(g.lam_num, g.lam_den, p)),
                                   Bc.ctypes.data, int(level), R.ctypes.data), "pleiden_refine")
    return R[:g.n]


def rand(seed: int, level: int, stream: int, c: int) -> int:
    """The counter-based generator of pLeidenR (SplitMix64 output function)."""
    return int(_load().orc_rand(seed & 0xFFFFFFFF, level, stream, c))


def _run(g, params, trace, trace_passes, fn, extra=None):
    p = params or Params()
    h = _graph(g)
    labels = np.zeros(max(g.n, 1), dtype=np.int32)
    res = _Result()
    cp = _c_params(g.lam_num, g.lam_den, p)
    rec = _Recorder(passes=trace_passes)
    cb = _CB(rec) if (trace or trace_passes) else _CB(0)
    lib = _load()
    if fn == "louvain_plus":
        rc = lib.orc_louvain_plus(ctypes.byref(h.g), ctypes.byref(cp), labels.ctypes.data,
                                  ctypes.byref(res), cb, None)
    elif fn == "louvain_plus_constrained":
        rc = lib.orc_louvain_plus_constrained(ctypes.byref(h.g), ctypes.byref(cp),
                                              extra.ctypes.data if extra.size else None,
                                              labels.ctypes.data, ctypes.byref(res), cb, None)
    elif fn == "pleiden":
        rc = lib.orc_pleiden(ctypes.byref(h.g), ctypes.byref(cp),
                             None if extra is None or not extra.size else extra.ctypes.data,
                             labels.ctypes.data, ctypes.byref(res), cb, None)
    else:
        rc = lib.orc_louvain_plus_iterated(ctypes.byref(h.g), ctypes.byref(cp), int(extra),
                                           labels.ctypes.data, ctypes.byref(res), cb, None)
    _rc(rc, fn)
    labels = labels[:g.n]
    out = {"n_clusters": res.n_clusters, "levels": res.levels, "passes_total": res.passes_total,
           "phi": _i128(res.phi_hi, res.phi_lo), "objective": res.objective,
           "modularity": res.modularity}
    return labels, out, rec.events
