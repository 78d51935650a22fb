"""Pins for the VIF oracle (Sect. 4.3, oracle/vif.py) against the exact GP
likelihood, plain Vecchia, FITC (Sect. 4.2) and the dense Sigma~_VIF."""
import numpy as np
import pytest

import oracle
import oracle.vif as vif
import synthetic_inputs as si


def setup(n_st=40, n_days=5, k=12, seed=1, order="time"):
    st = si.stations_uniform(n_st, seed)
    xy, t = si.station_days(st, n_days)
    perm = si.time_stratified_order(t, seed) if order == "time" else si.random_order(t.shape[0], seed)
    xy, t = np.ascontiguousarray(xy[perm]), np.ascontiguousarray(t[perm])
    th = oracle.theta_from_ranges(1.0, 0.2, 2.0, 0.5, 0.05)
    # inducing points: plain kMeans++ on scaled space-time coordinates
    X = np.concatenate([xy / 0.2, (t / 2.0)[:, None]], axis=1)
    C = si.kmeanspp(X, k, seed, lloyd_iters=10) if k else np.zeros((0, 3))
    xyk, tk = np.ascontiguousarray(C[:, :2] * 0.2), np.ascontiguousarray(C[:, 2] * 2.0)
    y = oracle.dense_sample(xy, t, th, si.standard_normal(t.shape[0], seed + 5))
    return xy, t, th, xyk, tk, y


def dense_nll(S, y):
    sign, ld = np.linalg.slogdet(S)
    assert sign > 0
    return 0.5 * y.shape[0] * np.log(2 * np.pi) + 0.5 * ld + 0.5 * y @ np.linalg.solve(S, y)


def test_all_predecessors_is_exact_for_any_k():
    # m = n-1: the residual's Vecchia factorisation is exact, so
    # Sigma~_VIF = U U^T + R + sigma^2 I = Sigma + sigma^2 I
    xy, t, th, xyk, tk, y = setup(n_st=30, n_days=4, k=15)
    U, r = vif.lowrank(xy, t, xyk, tk, th)
    m, nn, cnt = oracle.all_predecessors(t.shape[0])
    v = vif.nll(xy, t, th, U, m, nn, cnt, y)
    assert abs(v - oracle.dense_nll(xy, t, th, y)) / t.shape[0] < 1e-11


def test_k0_reduces_to_plain_vecchia():
    xy, t, th, xyk, tk, y = setup(k=0)
    U, r = vif.lowrank(xy, t, None, None, th)
    nn, cnt, rm, rm1 = vif.knn(xy, t, th, U, r, 8)
    nn_p, cnt_p, _, _ = oracle.knn(xy, t, th, 8)
    assert np.array_equal(nn, nn_p) and np.array_equal(cnt, cnt_p)
    assert vif.nll(xy, t, th, U, 8, nn, cnt, y) == pytest.approx(oracle.nll(xy, t, th, 8, nn, cnt, y), rel=1e-12)


def test_m0_reduces_to_fitc():
    # FITC (Sect. 4.2): Sigma_nk Sigma_kk^{-1} Sigma_kn + diag(Sigma - that) + sigma^2 I
    xy, t, th, xyk, tk, y = setup(k=10)
    n = t.shape[0]
    Skk = oracle.cov_matrix(xyk, tk, xyk, tk, th)
    Snk = oracle.cov_matrix(xy, t, xyk, tk, th)
    low = Snk @ np.linalg.solve(Skk, Snk.T)
    S = low + np.diag(th[0] - np.diag(low)) + th[4] * np.eye(n)
    U, r = vif.lowrank(xy, t, xyk, tk, th)
    nn = np.zeros((n, 0), dtype=np.int32)
    cnt = np.zeros(n, dtype=np.int32)
    assert abs(vif.nll(xy, t, th, U, 0, nn, cnt, y) - dense_nll(S, y)) / n < 1e-11


@pytest.mark.parametrize("order", ["time", "random"])
def test_woodbury_matches_dense_sigma(order):
    xy, t, th, xyk, tk, y = setup(k=12, order=order)
    U, r = vif.lowrank(xy, t, xyk, tk, th)
    assert np.all(r > 0)
    nn, cnt, rm, rm1 = vif.knn(xy, t, th, U, r, 6)
    A, D = vif.factor(xy, t, th, U, 6, nn, cnt)
    assert np.all(D >= th[4] * (1 - 1e-12))
    S = vif.dense_sigma(xy, t, th, U, 6, nn, cnt, A, D)
    v = vif.nll(xy, t, th, U, 6, nn, cnt, y, A, D)
    assert abs(v - dense_nll(S, y)) / t.shape[0] < 1e-11


def test_residual_neighbours_match_python_sort():
    xy, t, th, xyk, tk, y = setup(n_st=20, n_days=4, k=8, order="random")
    U, r = vif.lowrank(xy, t, xyk, tk, th)
    nn, cnt, _, _ = vif.knn(xy, t, th, U, r, 5)
    n = t.shape[0]
    C = oracle.cov_matrix(xy, t, xy, t, th)
    R = C - U @ U.T
    tiny = 1e-12 * th[0]
    for i in range(n):
        rho = [abs(R[i, j]) / np.sqrt(R[i, i] * R[j, j]) if min(r[i], r[j]) > tiny else 0.0 for j in range(i)]
        ref = sorted(range(i), key=lambda j: (-rho[j], j))[:5]
        assert list(nn[i, :cnt[i]]) == ref
    # the residual is a covariance: |rho| <= 1
    keep = r > tiny
    d = np.sqrt(np.diag(R)[keep])
    assert np.all(np.abs(R[np.ix_(keep, keep)] / d[:, None] / d[None, :]) <= 1 + 1e-9)
    assert np.all(r >= -1e-12)


def _vif_nll_at(xy, t, th, xyk, tk, m, nn, cnt, y):
    U, _ = vif.lowrank(xy, t, xyk, tk, th)
    return vif.nll(xy, t, th, U, m, nn, cnt, y)


def test_gradient_matches_central_differences():
    # d NLL / d theta_j against (NLL(theta + h e_j) - NLL(theta - h e_j)) / 2h,
    # h relative 1e-5: the truncation error is O(h^2) ~ 1e-10 relative
    xy, t, th, xyk, tk, y = setup(n_st=16, n_days=4, k=10, order="random")
    U, r = vif.lowrank(xy, t, xyk, tk, th)
    nn, cnt, _, _ = vif.knn(xy, t, th, U, r, 5)
    v, g = vif.nll_grad(xy, t, th, xyk, tk, 5, nn, cnt, y)
    assert v == pytest.approx(vif.nll(xy, t, th, U, 5, nn, cnt, y), rel=1e-12)
    for j in range(5):
        h = 1e-5 * th[j]
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        fd = (_vif_nll_at(xy, t, tp, xyk, tk, 5, nn, cnt, y) - _vif_nll_at(xy, t, tm, xyk, tk, 5, nn, cnt, y)) / (2 * h)
        assert g[j] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(g).max()), j


def test_gradient_k0_is_plain_vecchia_gradient():
    xy, t, th, xyk, tk, y = setup(n_st=16, n_days=4, k=0)
    nn, cnt, _, _ = oracle.knn(xy, t, th, 6)
    v, g = vif.nll_grad(xy, t, th, None, None, 6, nn, cnt, y)
    v0, g0 = oracle.nll_grad(xy, t, th, 6, nn, cnt, y)
    assert v == pytest.approx(v0, rel=1e-12)
    np.testing.assert_allclose(g, g0, rtol=1e-9, atol=1e-10 * np.abs(g0).max())


def test_gradient_all_predecessors_is_exact_gp_gradient():
    # m = n-1: Sigma~_VIF = Sigma + sigma^2 I for every theta, so the gradient
    # is the exact GP gradient whatever the inducing points
    xy, t, th, xyk, tk, y = setup(n_st=12, n_days=4, k=9)
    m, nn, cnt = oracle.all_predecessors(t.shape[0])
    v, g = vif.nll_grad(xy, t, th, xyk, tk, m, nn, cnt, y)
    v0, g0 = oracle.dense_nll(xy, t, th, y, grad=True)
    assert v == pytest.approx(v0, rel=1e-11)
    np.testing.assert_allclose(g, g0, rtol=1e-8, atol=1e-9 * np.abs(g0).max())


def test_gradient_variance_scaling_identity():
    # scaling sigma1^2 and the nugget by lambda scales Sigma_nk and Sigma_kk, so
    # U by sqrt(lambda), the residual and its factor's D_i by lambda, and leaves
    # A_i and the neighbour sets unchanged: Sigma~_VIF(lambda) = lambda
    # Sigma~_VIF, hence at lambda = 1
    #   sigma1^2 dNLL/dsigma1^2 + sigma^2 dNLL/dsigma^2 = n/2 - y^T Sigma~_VIF^{-1} y / 2
    # (y^T Sigma~_VIF^{-1} y from the densely formed matrix)
    xy, t, th, xyk, tk, y = setup(n_st=16, n_days=4, k=10, order="random")
    n = t.shape[0]
    U, r = vif.lowrank(xy, t, xyk, tk, th)
    nn, cnt, _, _ = vif.knn(xy, t, th, U, r, 5)
    _, g = vif.nll_grad(xy, t, th, xyk, tk, 5, nn, cnt, y)
    S = vif.dense_sigma(xy, t, th, U, 5, nn, cnt)
    rhs = 0.5 * n - 0.5 * y @ np.linalg.solve(S, y)
    lhs = th[0] * g[0] + th[4] * g[4]
    assert lhs == pytest.approx(rhs, rel=1e-9, abs=1e-9 * n)
    # the same with the FITC special case (m = 0)
    nn0 = np.zeros((n, 0), dtype=np.int32)
    cnt0 = np.zeros(n, dtype=np.int32)
    _, g0 = vif.nll_grad(xy, t, th, xyk, tk, 0, nn0, cnt0, y)
    S0 = vif.dense_sigma(xy, t, th, U, 0, nn0, cnt0)
    assert th[0] * g0[0] + th[4] * g0[4] == pytest.approx(0.5 * n - 0.5 * y @ np.linalg.solve(S0, y), rel=1e-9,
                                                          abs=1e-9 * n)


def test_lowrank_rows_and_knn_rows_match_the_whole_matrix_versions():
    # the chunked low rank and the per-row search are the same definitions
    # evaluated piecewise: identical to lowrank() and knn() on a small case
    rng = np.random.default_rng(3)
    xy = rng.random((300, 2))
    t = rng.integers(0, 6, 300).astype(float)
    th = oracle.theta_from_ranges(1.0, 0.2, 2.0, 0.5, 0.05)
    xyk = rng.random((12, 2))
    tk = rng.integers(0, 6, 12).astype(float)
    U, r = vif.lowrank(xy, t, xyk, tk, th)
    U2, r2 = vif.lowrank_rows(xy, t, xyk, tk, th, chunk=64, threads=3)
    np.testing.assert_allclose(U2, U, rtol=0, atol=1e-14)
    np.testing.assert_allclose(r2, r, rtol=0, atol=1e-14)
    nn, cnt, rm, rm1 = vif.knn(xy, t, th, U, r, 7)
    rows = np.array([0, 1, 5, 8, 150, 299])
    nn2, cnt2, rm2, rm12 = vif.knn_rows(xy, t, th, U, r, 7, rows)
    assert np.array_equal(nn2, nn[rows]) and np.array_equal(cnt2, cnt[rows])
    np.testing.assert_array_equal(rm2, rm[rows])
    np.testing.assert_array_equal(rm12, rm1[rows])
