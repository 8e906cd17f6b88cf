"""The in-place update of kept tables (CPU, no GPU).

With opts.tables = 1 the CUDA path keeps each high-degree vertex's table
S(v, .) across the passes of a LocalMovePasses call and, instead of
re-aggregating, applies the last pass's moves to it (Section IV-A-3,
Algorithm 2's update of the affected tables): a mover v from X to Y takes
w(u, v) from S(u, X) and adds it to S(u, Y) for every neighbour u, keys are
never deleted, and a sum of 0 means "no longer adjacent".  Here that rule,
run on every vertex over the oracle's passes, must give exactly the tables
recomputed from the labels entering each pass, including moves to new empty
clusters whose ids were freed in the same pass."""
import collections

import numpy as np
import pytest

import graphgen as gg
import oracle


def tables_from(rp, col, ew, C):
    T = []
    for v in range(rp.shape[0] - 1):
        t = collections.Counter()
        for e in range(rp[v], rp[v + 1]):
            t[int(C[col[e]])] += int(ew[e])
        T.append(t)
    return T


def apply_moves(T, rp, col, ew, C0, C1, moved):
    for v in np.nonzero(moved)[0]:
        xo, xn = int(C0[v]), int(C1[v])
        for e in range(rp[v], rp[v + 1]):
            u = col[e]
            T[u][xo] -= int(ew[e])  # the key stays, possibly at 0
            T[u][xn] += int(ew[e])


def adjacent(t):
    return {x: s for x, s in t.items() if s != 0}


def graph(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(10, 70))
    rp, col, ew = gg.random_graph(n, float(rng.uniform(0.05, 0.4)), seed, wmax=int(rng.integers(1, 6)))
    if seed % 2:
        return gg.cpm_inputs(rp, col, ew, 1, int(rng.integers(2, 12)))
    return gg.modularity_inputs(rp, col, ew)


@pytest.mark.parametrize("seed", range(16))
def test_updated_tables_equal_recomputed_tables(seed):
    g = graph(seed)
    _, _, ev = oracle.louvain_plus(g, trace=True, trace_passes=True)
    levels = {0: (g.row_ptr, g.col, g.ew)}
    for e in ev:
        if e["kind"] == "contract":
            levels[e["level"] + 1] = (e["row_ptr"], e["col"], e["ew"])
    T, prev, checked = None, None, 0
    for e in ev:
        if e["kind"] != "pass":
            continue
        rp, col, ew = levels[e["level"]]
        if e["pass"] == 1:  # a new LocalMovePasses call builds its tables
            T = tables_from(rp, col, ew, e["C_before"])
        else:
            apply_moves(T, rp, col, ew, prev["C_before"], prev["C"], prev["in_M"])
            fresh = tables_from(rp, col, ew, e["C_before"])
            assert all(adjacent(a) == adjacent(b) for a, b in zip(T, fresh)), (e["level"], e["phase"], e["pass"])
            assert all(s >= 0 for t in T for s in t.values())
            checked += 1
        prev = e
    assert checked > 0


def test_a_sum_of_zero_is_not_a_candidate():
    """Two vertices leave a cluster of three: the third vertex's table
    keeps the old key at 0, which must not count as an adjacent cluster."""
    rp, col, ew = gg.from_edges(3, np.array([0, 0]), np.array([1, 2]))
    T = tables_from(rp, col, ew, np.array([0, 0, 0]))
    apply_moves(T, rp, col, ew, np.array([0, 0, 0]), np.array([0, 1, 2]), np.array([False, True, True]))
    assert T[0][0] == 0 and adjacent(T[0]) == {1: 1, 2: 1}
