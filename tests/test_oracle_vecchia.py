"""Pins for the oracle's Vecchia factor, likelihood and gradient (Sect. 4.1,
Sect. 3.1) against numpy's dense linear algebra, exactness at m = n-1,
finite differences and closed-form identities."""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si


def small_problem(n_st=30, n_days=5, seed=0, rs=0.15, rt=2.0, gamma=0.5, nugget=0.05, nu=1.5, order="random"):
    st = si.stations_uniform(n_st, seed)
    xy, t = si.station_days(st, n_days)
    perm = si.random_order(t.shape[0], seed) if order == "random" else si.time_stratified_order(t, seed)
    xy, t = xy[perm], t[perm]
    th = oracle.theta_from_ranges(1.0, rs, rt, gamma, nugget, 0.4, 0.2, nu)
    return np.ascontiguousarray(xy), np.ascontiguousarray(t), th


def numpy_dense(xy, t, th, y):
    """Exact NLL and its gradient with numpy (Sect. 3.1): slogdet/solve/inv on the
    dense covariance; dSigma from the oracle's pinned covariance derivative."""
    n = t.shape[0]
    S = oracle.cov_matrix(xy, t, xy, t, th) + th[4] * np.eye(n)
    sign, logdet = np.linalg.slogdet(S)
    assert sign > 0
    alpha = np.linalg.solve(S, y)
    nll = 0.5 * n * np.log(2 * np.pi) + 0.5 * logdet + 0.5 * y @ alpha
    Sinv = np.linalg.inv(S)
    g = np.zeros(5)
    dS = np.zeros((4, n, n))
    for i in range(n):
        for j in range(n):
            h = np.hypot(*(xy[i] - xy[j]))
            dS[:, i, j] = oracle.cov_grad(th, h, t[i] - t[j])
    for p in range(4):
        g[p] = 0.5 * np.sum(Sinv * dS[p]) - 0.5 * alpha @ dS[p] @ alpha
    g[4] = 0.5 * np.trace(Sinv) - 0.5 * alpha @ alpha
    return nll, g


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_dense_oracle_matches_numpy(nu):
    xy, t, th = small_problem(n_st=25, n_days=4, nu=nu)
    y = oracle.dense_sample(xy, t, th, si.standard_normal(t.shape[0], 3))
    v, g = oracle.dense_nll(xy, t, th, y, grad=True)
    rv, rg = numpy_dense(xy, t, th, y)
    assert v == pytest.approx(rv, rel=1e-11)
    np.testing.assert_allclose(g, rg, rtol=1e-8, atol=1e-8)


@pytest.mark.parametrize("nu", [0.5, 1.5])
def test_vecchia_all_predecessors_is_exact(nu):
    # With N(i) = all predecessors the Vecchia factorisation is the exact chain
    # rule of the joint density (Sect. 4.1): NLL and gradient equal the dense ones.
    xy, t, th = small_problem(n_st=30, n_days=4, nu=nu)
    n = t.shape[0]
    y = oracle.dense_sample(xy, t, th, si.standard_normal(n, 4))
    m, nn, cnt = oracle.all_predecessors(n)
    v, g = oracle.nll_grad(xy, t, th, m, nn, cnt, y)
    rv, rg = numpy_dense(xy, t, th, y)
    assert abs(v - rv) / n <= 1e-12
    np.testing.assert_allclose(g, rg, rtol=1e-8, atol=1e-8)
    # the factor reproduces Sigma~ = B^{-1} D B^{-T} exactly
    A, D = oracle.factor(xy, t, th, m, nn, cnt)
    B = np.eye(n)
    for i in range(n):
        B[i, nn[i, :cnt[i]]] = -A[i, :cnt[i]]
    Binv = np.linalg.inv(B)
    S = oracle.cov_matrix(xy, t, xy, t, th) + th[4] * np.eye(n)
    np.testing.assert_allclose(Binv @ np.diag(D) @ Binv.T, S, atol=1e-10)


def test_gradient_central_differences():
    w = si.tiny_uniform(m=10)
    keep = 600
    xy, t = w.xy[:keep], w.t[:keep]
    th = oracle.theta_native(w.theta)
    nn, cnt, _, _ = oracle.knn(xy, t, th, 10)
    y = oracle.dense_sample(xy, t, th, w.z[:keep])
    v, g = oracle.nll_grad(xy, t, th, 10, nn, cnt, y)
    assert v == pytest.approx(oracle.nll(xy, t, th, 10, nn, cnt, y), rel=1e-14)
    for p in range(5):
        e = 1e-6 * max(1.0, abs(th[p]))
        tp, tm = th.copy(), th.copy()
        tp[p] += e
        tm[p] -= e
        fd = (oracle.nll(xy, t, th * 0 + tp, 10, nn, cnt, y) - oracle.nll(xy, t, tm, 10, nn, cnt, y)) / (2 * e)
        assert g[p] == pytest.approx(fd, rel=2e-6, abs=1e-5), p


def test_identities_and_bounds():
    w = si.tiny_uniform(m=10)
    xy, t, th, m = w.xy, w.t, oracle.theta_native(w.theta), 10
    n = t.shape[0]
    nn, cnt, _, _ = oracle.knn(xy, t, th, m)
    A, D = oracle.factor(xy, t, th, m, nn, cnt)
    # conditioning cannot remove the nugget nor add variance: sigma^2 <= D_i <= sigma1^2 + sigma^2
    assert np.all(D >= th[4] * (1 - 1e-12)) and np.all(D <= (th[0] + th[4]) * (1 + 1e-12))
    assert D[0] == pytest.approx(th[0] + th[4], rel=1e-15)  # row 0 has no neighbours
    # whitening identity: y drawn by Vecchia sampling with the same (nn, theta) has
    # e_i = z_i, so NLL = n/2 log 2pi + 1/2 sum log D_i + 1/2 sum z_i^2
    z = w.z
    y = oracle.vecchia_sample(m, nn, cnt, A, D, z)
    v, terms = oracle.nll(xy, t, th, m, nn, cnt, y, terms=True)
    ref = 0.5 * n * np.log(2 * np.pi) + 0.5 * np.log(D).sum() + 0.5 * (z ** 2).sum()
    assert abs(v - ref) / n < 1e-13
    np.testing.assert_allclose(terms, 0.5 * np.log(D) + 0.5 * z ** 2, rtol=1e-11, atol=1e-12)
    # variance scaling identity: scaling sigma1^2 and sigma^2 by lambda scales every
    # D_i by lambda and leaves A_i unchanged, hence
    # sigma1^2 dNLL/dsigma1^2 + sigma^2 dNLL/dsigma^2 = n/2 - 1/2 sum e_i^2
    y2 = oracle.dense_sample(xy, t, th, si.standard_normal(n, 9))
    _, g = oracle.nll_grad(xy, t, th, m, nn, cnt, y2)
    r = y2 - np.array([A[i, :cnt[i]] @ y2[nn[i, :cnt[i]]] for i in range(n)])
    e2 = (r ** 2 / D).sum()
    assert th[0] * g[0] + th[4] * g[4] == pytest.approx(n / 2 - 0.5 * e2, rel=1e-10)


def py_knn(xy, t, th, m):
    """Neighbour selection written as a sort over all predecessors (Sect. 4.4.1)."""
    n = t.shape[0]
    C = oracle.cov_matrix(xy, t, xy, t, th)
    out = []
    for i in range(n):
        rho = [abs(C[i, j]) / np.sqrt(C[i, i] * C[j, j]) for j in range(i)]
        order = sorted(range(i), key=lambda j: (-rho[j], j))
        out.append(order[:m])
    return out


@pytest.mark.parametrize("order", ["random", "time"])
def test_knn_matches_python_sort(order):
    xy, t, th = small_problem(n_st=40, n_days=6, order=order)
    m = 7
    nn, cnt, rm, rm1 = oracle.knn(xy, t, th, m)
    ref = py_knn(xy, t, th, m)
    for i in range(t.shape[0]):
        assert cnt[i] == min(i, m)
        assert list(nn[i, :cnt[i]]) == ref[i]
        assert np.all(nn[i, cnt[i]:] == -1)


def test_knn_exact_ties_pick_smaller_index():
    # the same station observed on days 0 and 2 is equally correlated with a
    # query on day 1 at that station: the tie goes to the smaller index
    xy = np.array([[0.5, 0.5], [0.5, 0.5], [0.1, 0.9], [0.5, 0.5]])
    t = np.array([2.0, 0.0, 1.0, 1.0])
    th = oracle.theta_from_ranges(1.0, 0.1, 3.0, 0.5, 0.05)
    nn, cnt, rm, rm1 = oracle.knn(xy, t, th, 1)
    assert nn[3, 0] == 0
    assert rm[3] == rm1[3]
    assert 3 in oracle.tie_rows(rm, rm1)


def test_cond_estimate_closed_form_and_bounds():
    # two points: the block [[s, c], [c, s]] (s = sigma1^2 + nugget, c the
    # covariance) has pivots sqrt(s) and sqrt(s - c^2 / s), so the estimate
    # (max L_jj / min L_jj)^2 is s^2 / (s^2 - c^2)
    th = oracle.theta_from_ranges(1.0, 0.1, 3.0, 0.5, 0.05)
    xy = np.array([[0.3, 0.4], [0.33, 0.38]])
    t = np.array([2.0, 3.0])
    c = oracle.cov(th, float(np.hypot(0.03, 0.02)), 1.0)
    s = th[0] + th[4]
    est = oracle.cond_estimates(xy, t, th, np.array([[-1], [0]], dtype=np.int32), np.array([0, 1], dtype=np.int32))
    assert est[0] == 1.0
    assert est[1] == pytest.approx(s * s / (s * s - c * c), rel=1e-12)
    # larger blocks: each squared pivot is a Schur complement, which lies
    # between the extreme eigenvalues, so 1 <= estimate <= cond_2(block)
    w = si.tiny_uniform(m=10)
    nn, cnt, _, _ = oracle.knn(w.xy, w.t, th, w.m)
    rows = np.arange(20, 2000, 97)
    est = oracle.cond_estimates(w.xy, w.t, th, nn, cnt, rows)
    for q, i in enumerate(rows):
        idx = np.concatenate([nn[i][:cnt[i]], [i]])
        K = oracle.cov_matrix(w.xy[idx], w.t[idx], w.xy[idx], w.t[idx], th) + th[4] * np.eye(idx.shape[0])
        ev = np.linalg.eigvalsh(K)
        assert 1.0 < est[q] <= ev[-1] / ev[0] * (1 + 1e-9)
