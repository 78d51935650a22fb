"""Pins of the Vecchia prediction oracle (oracle/predict.py) against what the
paper and the mathematics fix, without the GPU."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import oracle.predict as opred
import synthetic_inputs as si


def small(n_st=12, n_days=5, seed=3):
    st = si.stations_uniform(n_st, seed)
    xy, t = si.station_days(st, n_days)
    order = si.random_order(t.shape[0], seed)
    xy, t = np.ascontiguousarray(xy[order]), np.ascontiguousarray(t[order])
    th = oracle.theta_from_ranges(1.0, 0.2, 3.0, 0.5, 0.05)
    y = oracle.dense_sample(xy, t, th, si.standard_normal(t.shape[0], seed + 1))
    rng = np.random.default_rng(seed + 2)
    xyp = rng.random((25, 2))
    tp = rng.integers(-1, n_days + 2, 25).astype(float)
    return xy, t, y, xyp, tp, th


def test_all_neighbours_is_exact_kriging():
    # m = n: the predictive mean and variance of Sect. 3.1, from one Cholesky
    # factor of the full training covariance
    xy, t, y, xyp, tp, th = small()
    n = t.shape[0]
    K = oracle.cov_matrix(xy, t, xy, t, th) + th[4] * np.eye(n)
    cf = sla.cho_factor(K, lower=True)
    Kp = oracle.cov_matrix(xy, t, xyp, tp, th)            # n x np
    mean_ref = Kp.T @ sla.cho_solve(cf, y)
    V = sla.solve_triangular(cf[0], Kp, lower=True)
    var_ref = th[0] + th[4] - (V * V).sum(0)
    mean, var, _ = opred.predict(xy, t, y, xyp, tp, th, n)
    np.testing.assert_allclose(mean, mean_ref, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(var, var_ref, rtol=1e-9, atol=1e-11)
    _, var_lat, _ = opred.predict(xy, t, y, xyp, tp, th, n, latent=True)
    np.testing.assert_allclose(var_lat, var_ref - th[4], rtol=1e-9, atol=1e-11)


def test_far_point_returns_the_prior_and_variances_are_bounded():
    xy, t, y, xyp, tp, th = small()
    xyp = np.concatenate([xyp, [[1e6, 1e6]]])
    tp = np.concatenate([tp, [1e6]])
    mean, var, _ = opred.predict(xy, t, y, xyp, tp, th, 8)
    assert abs(mean[-1]) < 1e-12 and abs(var[-1] - (th[0] + th[4])) < 1e-12
    assert np.all(var > 0) and np.all(var <= th[0] + th[4] + 1e-12)


def test_neighbours_are_the_most_correlated_training_points():
    xy, t, y, xyp, tp, th = small()
    m = 7
    nn, cnt = opred.neighbours(xy, t, xyp, tp, th, m)
    R = oracle.cov_matrix(xyp, tp, xy, t, th) / th[0]
    for p in range(tp.shape[0]):
        sel = nn[p, :cnt[p]]
        r_sel = R[p, sel]
        assert np.all(np.diff(r_sel) <= 0)                 # decreasing
        rest = np.setdiff1d(np.arange(t.shape[0]), sel)
        assert R[p, rest].max() <= r_sel.min()             # nothing better left out


def test_no_training_points():
    xy, t, y, xyp, tp, th = small()
    mean, var, nn = opred.predict(xy[:0], t[:0], y[:0], xyp, tp, th, 5)
    assert np.all(mean == 0) and np.allclose(var, th[0] + th[4]) and np.all(nn == -1)
