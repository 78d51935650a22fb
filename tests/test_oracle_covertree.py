"""Pins of the oracle's cover-tree search (Algorithms 1 and 2 of Sect. 4.4.1)
against its brute-force search and the tree's construction invariants."""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si


def problem(n_st, n_days, seed, order, rs=0.1, rt=3.0, nu=1.5, jitter=0.0):
    st = si.stations_uniform(n_st, seed)
    xy, t = si.station_days(st, n_days)
    if jitter:
        t = t + jitter * np.random.default_rng(seed).random(t.shape[0])
    perm = si.random_order(t.shape[0], seed) if order == "random" else si.time_stratified_order(t, seed)
    th = oracle.theta_from_ranges(1.0, rs, rt, 0.5, 0.05, 0.4, 0.2, nu)
    return np.ascontiguousarray(xy[perm]), np.ascontiguousarray(t[perm]), th


@pytest.mark.parametrize("case", [
    dict(n_st=200, n_days=10, seed=0, order="random", m=10),
    dict(n_st=150, n_days=20, seed=1, order="time", m=20),
    dict(n_st=100, n_days=12, seed=2, order="time", m=31, rs=0.3, rt=8.0, nu=0.5),
    dict(n_st=120, n_days=8, seed=3, order="random", m=5, nu=2.5, jitter=0.4),
    # long ranges: high correlations, a deep tree whose pruning radius matters
    # (a radius of 2^-(j+3) instead of 2^-(j-1) loses neighbours here)
    dict(n_st=200, n_days=10, seed=5, order="random", m=10, rs=0.8, rt=40.0),
    dict(n_st=300, n_days=6, seed=6, order="time", m=10, rs=2.0, rt=100.0),
    dict(n_st=400, n_days=5, seed=7, order="random", m=10, rs=5.0, rt=200.0, nu=0.5),
])
def test_cover_tree_search_equals_brute_force(case):
    m = case.pop("m")
    xy, t, th = problem(**case)
    with oracle.CoverTree(xy, t, th) as T:
        assert T.depth >= 3
        got = T.knn(m)
    ref = oracle.knn(xy, t, th, m)
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g, r)


def test_cover_tree_invariants():
    xy, t, th = problem(150, 10, 4, "time")
    n = t.shape[0]
    with oracle.CoverTree(xy, t, th) as T:
        level, parent = T.structure()
        depth = T.depth
    # every point is a knot of exactly one level; point 0 is the root
    assert level[0] == 1 and parent[0] == -1
    assert np.all(level[1:] >= 2) and level.max() <= depth
    # children come after their knot and sit one level below it
    kids = np.arange(1, n)
    assert np.all(parent[kids] < kids) and np.all(parent[kids] >= 0)
    assert np.all(level[kids] == level[parent[kids]] + 1)
    # a knot of level L >= 2 covers its subtree within d_c <= 2^-(L-1)
    for c in kids:
        p = parent[c]
        L = level[p]
        if L < 2:
            continue
        h = float(np.hypot(*(xy[c] - xy[p])))
        rho = abs(oracle.cov(th, h, t[c] - t[p])) / th[0]
        assert np.sqrt(max(0.0, 1.0 - rho)) <= 2.0 ** -(L - 1) * (1 + 1e-12)
