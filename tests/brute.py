"""Brute-force restatements used to pin the oracle (pure numpy, tiny graphs).

Nothing here calls the oracle.  Each function is the plain definition from
the paper, evaluated by exhaustion:

* ``pair_objective``: Eq. 1 first form, Lambda * sum over ordered pairs
  u != v in the same cluster of (w(u,v) - lambda w(u) w(v)), from a dense
  weight matrix.
* ``move``: apply one vertex move (a new empty cluster gets a fresh label).
* ``set_partitions``: every partition of {0..n-1} as restricted growth strings.
* ``coarse_dense``: the coarse adjacency P^T A P (off-diagonal) for a
  membership matrix P, the coarse graph of Section III-A.
"""
from __future__ import annotations

import numpy as np


def dense(rp, col, ew) -> np.ndarray:
    n = rp.shape[0] - 1
    A = np.zeros((n, n), dtype=np.int64)
    rows = np.repeat(np.arange(n), np.diff(rp))
    A[rows, col] = ew
    return A


def pair_matrix(A: np.ndarray, vw: np.ndarray, mu: int, Lam: int) -> np.ndarray:
    """Lambda * w'(u, v) = Lambda w(u,v) - mu w(u) w(v) for u != v, 0 on the diagonal."""
    P = Lam * A - mu * np.outer(vw, vw)
    np.fill_diagonal(P, 0)
    return P


def pair_objective(P: np.ndarray, labels) -> int:
    lab = np.asarray(labels)
    same = lab[:, None] == lab[None, :]
    return int((P * same).sum())


def move(labels, v: int, X: int, empty: int = -2) -> np.ndarray:
    lab = np.array(labels, dtype=np.int64, copy=True)
    lab[v] = (lab.max() + 1 + v) if X == empty else X
    return lab


def set_partitions(n: int) -> np.ndarray:
    """All set partitions of n items as restricted growth strings (Bell(n) rows)."""
    out = []
    a = [0] * n

    def rec(i, m):
        if i == n:
            out.append(a.copy())
            return
        for c in range(m + 1):
            a[i] = c
            rec(i + 1, max(m, c + 1))

    if n == 0:
        return np.zeros((1, 0), dtype=np.int64)
    a[0] = 0
    rec(1, 1)
    return np.array(out, dtype=np.int64)


def best_partition_objective(P: np.ndarray) -> int:
    n = P.shape[0]
    R = set_partitions(n)
    best = None
    for chunk in range(0, R.shape[0], 20000):
        r = R[chunk:chunk + 20000]
        same = r[:, :, None] == r[:, None, :]
        vals = (same * P[None, :, :]).sum(axis=(1, 2))
        m = int(vals.max())
        best = m if best is None else max(best, m)
    return best


def coarse_dense(A: np.ndarray, labels, n_c: int) -> np.ndarray:
    n = A.shape[0]
    Pm = np.zeros((n, n_c), dtype=np.int64)
    Pm[np.arange(n), np.asarray(labels)] = 1
    Ac = Pm.T @ A @ Pm
    np.fill_diagonal(Ac, 0)
    return Ac


def fmix32(h: int) -> int:
    """MurmurHash3 32-bit finaliser (Appleby, public domain)."""
    h = int(h) & 0xFFFFFFFF
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & 0xFFFFFFFF
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & 0xFFFFFFFF
    h ^= h >> 16
    return h
