"""Seeded synthetic graph inputs shared by the CPU oracle and the CUDA path.

This module is input infrastructure: it builds graphs and the per-workload
vertex weights and resolution, and holds none of the clustering arithmetic.
Every graph is an undirected CSR (``row_ptr`` int64[n+1], ``col`` int32[nnz],
``ew`` int32[nnz]) storing both directions of each edge, rows sorted, no
self-loops, no duplicates, positive integer weights (the graph model of
Section II of the paper).  The heavy generators are C (``graphgen.c``),
compiled in-tree with gcc on first use.

Workload recipes (seeded; the paper's 57-graph dataset is not used):

* ``sbm_planted``  planted-partition SBM, 10,000 vertices in 100 blocks,
  p_in 0.05, p_out 0.0005, unit weights, modularity, seed 0.
* ``rmat``         R-MAT scale 22, edge factor 16, (a,b,c,d)=(.57,.19,.19,.05),
  weights uniform in [1,8], modularity.
* ``grid_cpm``     3-D 7-point lattice 256^3 with 1% of edges rewired, weights
  in [1,16], unit vertex weights, CPM with lambda = 1/100.
* ``batched_sbms`` 4,096 SBMs with log-uniform sizes and block counts.
* tiny random graphs for the oracle pins.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libgraphgen.so")

GCC_FLAGS = ["-O2", "-std=c11", "-shared", "-fPIC", "-Wall", "-Wextra", "-Wno-unused-parameter"]


def build(force: bool = False) -> str:
    """Compile libgraphgen.so in-tree (gcc); returns its path."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp"
        subprocess.check_call(["gcc", *GCC_FLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _CSR(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("row_ptr", ctypes.POINTER(ctypes.c_int64)),
        ("col", ctypes.POINTER(ctypes.c_int32)),
        ("ew", ctypes.POINTER(ctypes.c_int32)),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, u64, i32, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double
        p = ctypes.POINTER(_CSR)
        lib.gg_sbm.argtypes = [i64, i64, dbl, dbl, u64, i32, i32, p]
        lib.gg_rmat.argtypes = [ctypes.c_int, i64, dbl, dbl, dbl, u64, i32, i32, p]
        lib.gg_grid3d.argtypes = [i64, i64, i64, dbl, u64, i32, i32, p]
        lib.gg_from_edges.argtypes = [i64, i64, ctypes.c_void_p, ctypes.c_void_p, u64, i32, i32, p]
        lib.gg_free.argtypes = [p]
        for f in (lib.gg_sbm, lib.gg_rmat, lib.gg_grid3d, lib.gg_from_edges):
            f.restype = ctypes.c_int
        lib.gg_free.restype = None
        _lib = lib
    return _lib


@dataclass
class Graph:
    """Undirected CSR graph plus the LambdaCC inputs of one workload."""

    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray      # int32[nnz]
    ew: np.ndarray       # int32[nnz]
    vw: np.ndarray = None  # int64[n]   vertex weights w(v)
    lam_num: int = 0     # lambda = lam_num / lam_den
    lam_den: int = 1
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])


def _take(csr: _CSR) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    n, nnz = csr.n, csr.nnz
    rp = np.ctypeslib.as_array(csr.row_ptr, shape=(n + 1,)).copy()
    if nnz > 0:
        col = np.ctypeslib.as_array(csr.col, shape=(nnz,)).copy()
        ew = np.ctypeslib.as_array(csr.ew, shape=(nnz,)).copy()
    else:
        col = np.zeros(0, np.int32)
        ew = np.zeros(0, np.int32)
    _load().gg_free(ctypes.byref(csr))
    return rp, col, ew


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"graphgen: {what} failed with code {rc}")


def sbm(n: int, nblocks: int, p_in: float, p_out: float, seed: int, wmin: int = 1, wmax: int = 1):
    csr = _CSR()
    _check(_load().gg_sbm(n, nblocks, p_in, p_out, seed, wmin, wmax, ctypes.byref(csr)), "sbm")
    return _take(csr)


def rmat_csr(scale: int, edge_factor: int = 16, a=0.57, b=0.19, c=0.19, seed: int = 1,
             wmin: int = 1, wmax: int = 8):
    csr = _CSR()
    _check(_load().gg_rmat(scale, edge_factor, a, b, c, seed, wmin, wmax, ctypes.byref(csr)), "rmat")
    return _take(csr)


def grid3d_csr(nx: int, ny: int, nz: int, rewire_p: float, seed: int, wmin: int = 1, wmax: int = 16):
    csr = _CSR()
    _check(_load().gg_grid3d(nx, ny, nz, rewire_p, seed, wmin, wmax, ctypes.byref(csr)), "grid3d")
    return _take(csr)


def from_edges(n: int, src, dst, seed: int = 0, wmin: int = 1, wmax: int = 1):
    src = np.ascontiguousarray(src, dtype=np.int64)
    dst = np.ascontiguousarray(dst, dtype=np.int64)
    csr = _CSR()
    _check(_load().gg_from_edges(n, src.shape[0], src.ctypes.data, dst.ctypes.data, seed, wmin, wmax,
                                 ctypes.byref(csr)), "from_edges")
    return _take(csr)


# ------------------------------------------------------ LambdaCC inputs ---

def weighted_degree(row_ptr: np.ndarray, ew: np.ndarray) -> np.ndarray:
    """w(v) = sum of incident edge weights (the modularity vertex weight)."""
    n = row_ptr.shape[0] - 1
    out = np.zeros(n, dtype=np.int64)
    if ew.shape[0]:
        seg = np.add.reduceat(ew.astype(np.int64), np.minimum(row_ptr[:-1], ew.shape[0] - 1))
        deg = np.diff(row_ptr)
        out = np.where(deg > 0, seg, 0).astype(np.int64)
    return out


def modularity_inputs(rp, col, ew, gamma_num: int = 1, gamma_den: int = 1, name: str = "") -> Graph:
    """Modularity as a LambdaCC instance: w(v) = weighted degree and
    lambda = gamma / (2 m_w), 2 m_w = total ordered edge weight."""
    vw = weighted_degree(rp, ew)
    two_m = int(ew.astype(np.int64).sum())
    return Graph(rp, col, ew, vw, gamma_num, gamma_den * max(two_m, 1), name,
                 {"objective": "modularity"})


def cpm_inputs(rp, col, ew, lam_num: int, lam_den: int, name: str = "") -> Graph:
    """Constant Potts model: unit vertex weights and a rational lambda."""
    n = rp.shape[0] - 1
    return Graph(rp, col, ew, np.ones(n, dtype=np.int64), lam_num, lam_den, name,
                 {"objective": "cpm"})


# ------------------------------------------------------------- recipes ---

def sbm_planted(n: int = 10_000, blocks: int = 100, p_in: float = 0.05, p_out: float = 0.0005,
                seed: int = 0) -> Graph:
    """Planted partition SBM with unit weights; modularity objective."""
    rp, col, ew = sbm(n, blocks, p_in, p_out, seed, 1, 1)
    g = modularity_inputs(rp, col, ew, name=f"sbm_n{n}_k{blocks}")
    g.meta.update(blocks=blocks, p_in=p_in, p_out=p_out, seed=seed)
    return g


def rmat(scale: int = 22, edge_factor: int = 16, seed: int = 1, wmax: int = 8) -> Graph:
    """R-MAT, symmetrised, deduplicated, loops removed, weights in [1, wmax]; modularity."""
    rp, col, ew = rmat_csr(scale, edge_factor, 0.57, 0.19, 0.19, seed, 1, wmax)
    g = modularity_inputs(rp, col, ew, name=f"rmat{scale}_ef{edge_factor}")
    g.meta.update(scale=scale, edge_factor=edge_factor, seed=seed)
    return g


def grid_cpm(side: int = 256, rewire: float = 0.01, seed: int = 2, wmax: int = 16,
             lam_num: int = 1, lam_den: int = 100) -> Graph:
    """3-D 7-point lattice side^3 with rewiring; CPM with lambda = lam_num/lam_den."""
    rp, col, ew = grid3d_csr(side, side, side, rewire, seed, 1, wmax)
    g = cpm_inputs(rp, col, ew, lam_num, lam_den, name=f"grid{side}^3_cpm")
    g.meta.update(side=side, rewire=rewire, seed=seed)
    return g


def batched_sbm_params(count: int, seed: int = 3, n_lo: int = 100, n_hi: int = 100_000,
                       k_lo: int = 2, k_hi: int = 500, d_lo: float = 4.0, d_hi: float = 32.0,
                       mixing: float = 0.5):
    """Per-graph (n, blocks, p_in, p_out, seed) for the batched workload:
    n and block count log-uniform, mean degree uniform, a fixed fraction
    `mixing` of each vertex's expected degree leaving its block."""
    rng = np.random.default_rng(seed)
    out = []
    for g in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        kmax = min(k_hi, n)
        k = int(round(math.exp(rng.uniform(math.log(k_lo), math.log(kmax)))))
        k = max(1, min(k, n))
        d = float(rng.uniform(d_lo, d_hi))
        s = n / k
        d_in = d * (1.0 - mixing)
        d_out = d * mixing
        p_in = min(1.0, d_in / max(s - 1.0, 1.0))
        p_out = min(1.0, d_out / max(n - s, 1.0)) if k > 1 else 0.0
        if k == 1:
            p_in = min(1.0, d / max(n - 1.0, 1.0))
        out.append((n, k, p_in, p_out, seed * 1_000_003 + g))
    return out


def expected_nnz(p) -> float:
    """Expected stored edges of one batched-recipe SBM (n, blocks, p_in, p_out, seed)."""
    n, k, p_in, p_out, _ = p
    s = n / k
    return n * (p_in * max(s - 1.0, 0.0) + p_out * (n - s))


def batched_sbms(count: int = 4096, seed: int = 3, threads: int | None = None,
                 indices=None, **kw) -> list[Graph]:
    """The batched workload's graphs (generated on `threads` host threads;
    each graph depends only on its own seed, so the result is the same).
    With `indices`, only those graphs of the workload, in that order."""
    import concurrent.futures as cf

    params = batched_sbm_params(count, seed, **kw)
    if indices is not None:
        params = [params[i] for i in indices]

    def one(p):
        n, k, p_in, p_out, s = p
        rp, col, ew = sbm(n, k, p_in, p_out, s, 1, 1)
        g = modularity_inputs(rp, col, ew, name=f"sbm_n{n}_k{k}")
        g.meta.update(blocks=k, p_in=p_in, p_out=p_out, seed=s)
        return g

    with cf.ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 4) as ex:
        return list(ex.map(one, params))


def served_request_params(count: int, seed: int = 4):
    """Per-request recipe of the served workload: 70% SBM (n log-uniform in
    [1e3, 1e6], blocks and degree as in the batched recipe), 30% R-MAT (scale
    uniform in 10..20, edge factor 16); weights uniform in [1, 8]; objective
    modularity or CPM lambda = 1/50 with probability 1/2 each."""
    rng = np.random.default_rng(seed)
    sbm_p = batched_sbm_params(count, seed=seed, n_lo=1_000, n_hi=1_000_000)
    out = []
    for r in range(count):
        kind = "sbm" if rng.random() < 0.7 else "rmat"
        cpm = bool(rng.random() < 0.5)
        scale = int(rng.integers(10, 21))
        out.append((kind, sbm_p[r] if kind == "sbm" else scale, cpm, seed * 1_000_003 + r))
    return out


def served_requests(count: int, seed: int = 4, threads: int | None = None) -> list[Graph]:
    """The served workload's request graphs, in arrival order."""
    import concurrent.futures as cf

    def one(p):
        kind, par, cpm, s = p
        if kind == "sbm":
            n, k, p_in, p_out, gs = par
            rp, col, ew = sbm(n, k, p_in, p_out, gs, 1, 8)
            name = f"sbm_n{n}_k{k}"
        else:
            rp, col, ew = rmat_csr(par, 16, 0.57, 0.19, 0.19, s, 1, 8)
            name = f"rmat{par}"
        if cpm:
            return cpm_inputs(rp, col, ew, 1, 50, name=name + "_cpm")
        return modularity_inputs(rp, col, ew, name=name + "_mod")

    with cf.ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 4) as ex:
        return list(ex.map(one, served_request_params(count, seed)))


def random_graph(n: int, p: float, seed: int, wmax: int = 1) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Tiny Erdos-Renyi G(n, p) built in numpy (seeded), weights in [1, wmax]."""
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.shape[0]) < p
    src, dst = iu[keep], ju[keep]
    return from_edges(n, src, dst, seed=seed, wmin=1, wmax=wmax)


def random_labels(n: int, k: int, seed: int) -> np.ndarray:
    """Seeded random clustering of n vertices into at most k labels (int32)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, max(k, 1), size=n).astype(np.int32)


def pack(graphs: list) -> dict:
    """Packs graphs into one CSR (disjoint union, global vertex ids) for the
    batched entry point: row_ptr, col, ew, vw, graph_ptr, lam_num, lam_den."""
    n_off, e_off = [0], [0]
    for g in graphs:
        n_off.append(n_off[-1] + g.n)
        e_off.append(e_off[-1] + g.nnz)
    rp = np.zeros(n_off[-1] + 1, dtype=np.int64)
    col = np.empty(e_off[-1], dtype=np.int32)
    ew = np.empty(e_off[-1], dtype=np.int32)
    vw = np.empty(n_off[-1], dtype=np.int64)
    for k, g in enumerate(graphs):
        rp[n_off[k] + 1:n_off[k + 1] + 1] = g.row_ptr[1:] + e_off[k]
        col[e_off[k]:e_off[k + 1]] = g.col + n_off[k]
        ew[e_off[k]:e_off[k + 1]] = g.ew
        vw[n_off[k]:n_off[k + 1]] = g.vw
    return {"row_ptr": rp, "col": col, "ew": ew, "vw": vw,
            "graph_ptr": np.array(n_off, dtype=np.int64),
            "lam_num": np.array([g.lam_num for g in graphs], dtype=np.int64),
            "lam_den": np.array([g.lam_den for g in graphs], dtype=np.int64)}
