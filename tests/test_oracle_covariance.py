"""Pins for the oracle's covariance (Eq. (2)) against facts the paper and the
mathematics fix: the printed effective ranges (Table A3, Sect. 6.1 and 6.2
parameter tables), scipy's Bessel K, and the reductions stated below Eq. (2)."""
import itertools
import math

import numpy as np
import pytest
import scipy.special as sp

import oracle
from conftest import golden


def theta(sigma1sq=1.0, c=10.0, a=1.0, gamma=0.5, nugget=0.05, alpha=0.4, delta=0.2, nu=1.5):
    return np.array([sigma1sq, c, a, gamma, nugget, alpha, delta, nu], dtype=np.float64)


def bisect(f, lo, hi, it=200):
    """root of a decreasing function on [lo, hi]"""
    for _ in range(it):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def space_range(th):
    s = th[0]
    hi = 1.0
    while oracle.cov(th, hi, 0.0) / s > 0.05:
        hi *= 2
    return bisect(lambda h: oracle.cov(th, h, 0.0) / s - 0.05, 0.0, hi)


def time_range(th):
    s = th[0]
    hi = 1.0
    while oracle.cov(th, 0.0, hi) / s > 0.05:
        hi *= 2
        if hi > 1e12:
            return math.inf
    return bisect(lambda u: oracle.cov(th, 0.0, u) / s - 0.05, 0.0, hi)


@pytest.mark.parametrize("nu", [0.5, 1.0, 1.5, 2.5, 0.8])
def test_matern_matches_bessel_k(nu):
    # M_nu(x) = 2^{1-nu}/Gamma(nu) x^nu K_nu(x): closed forms for nu in {.5,1.5,2.5}
    # must equal the general Bessel form (scipy's kv, an independent library).
    for x in [1e-3, 0.05, 0.3, 1.0, 2.0, 4.7439, 9.0, 20.0]:
        ref = 2 ** (1 - nu) / sp.gamma(nu) * x ** nu * sp.kv(nu, x)
        assert oracle.matern(nu, x) == pytest.approx(ref, rel=1e-12, abs=1e-300)
    assert oracle.matern(nu, 0.0) == 1.0


@pytest.mark.parametrize("row", golden("table_a3_effective_ranges.txt"), ids=lambda r: r[0])
def test_table_a3_effective_ranges(row):
    name, s1, a, c, alpha, nu, gamma, delta, tr, sr = row
    th = theta(float(s1), float(c), float(a), float(gamma), 0.0, float(alpha), float(delta), float(nu))
    t = time_range(th)
    if tr == "inf":
        assert t > 1e6  # alpha = 0.08: the 0.05 crossing lies beyond a million time units
    else:
        assert round(t, 2) == pytest.approx(float(tr), abs=1e-9)
    s = space_range(th)
    ndig = len(sr.split(".")[1])
    assert round(s, ndig) == pytest.approx(float(sr), abs=1e-9)


def _interval(fun, vals, halfulp):
    corners = [fun(*[v + d for v, d in zip(vals, ds)])
               for ds in itertools.product(*[(-h, h) for h in halfulp])]
    return min(corners), max(corners)


@pytest.mark.parametrize("row", golden("temperature_vif_params.txt"), ids=lambda r: r[0])
def test_temperature_table_ranges(row):
    # nu = 1.5; c per metre; space range printed in km, time in days
    _, nug, s1, a, c, alpha, gamma, delta, tr, sr, ok_t, ok_s = row
    a, c, alpha, gamma, delta = map(float, (a, c, alpha, gamma, delta))
    tfun = lambda a_, al_, g_, d_: time_range(theta(1.0, 1.0, a_, g_, 0.0, al_, d_, 1.5))
    lo, hi = _interval(tfun, (a, alpha, gamma, delta), (5e-4,) * 4)
    hit = lo <= float(tr) + 0.05 and hi >= float(tr) - 0.05
    assert hit == (ok_t == "1")
    sfun = lambda c_: space_range(theta(1.0, c_, 1.0, gamma, 0.0, alpha, delta, 1.5)) / 1e3
    lo, hi = _interval(sfun, (c,), (0.005e-6,))
    hit = lo <= float(sr) + 0.5 and hi >= float(sr) - 0.5
    assert hit == (ok_s == "1")


@pytest.mark.parametrize("row", golden("precipitation_vif_params.txt"), ids=lambda r: r[0])
def test_precipitation_table_ranges(row):
    # nu = 0.5 (exponential); c printed as c * 1e5 per metre
    _, s1, a, c5, alpha, gamma, delta, tr, sr, ok_t, ok_s = row
    a, c, alpha, gamma, delta = float(a), float(c5) * 1e-5, float(alpha), float(gamma), float(delta)
    tfun = lambda a_, al_, g_, d_: time_range(theta(1.0, 1.0, a_, g_, 0.0, al_, d_, 0.5))
    lo, hi = _interval(tfun, (a, alpha, gamma, delta), (5e-4,) * 4)
    assert (lo <= float(tr) + 0.05 and hi >= float(tr) - 0.05) == (ok_t == "1")
    sfun = lambda c_: space_range(theta(1.0, c_, 1.0, gamma, 0.0, alpha, delta, 0.5)) / 1e3
    lo, hi = _interval(sfun, (c,), (0.0005e-5,))
    assert (lo <= float(sr) + 0.5 and hi >= float(sr) - 0.5) == (ok_s == "1")


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_reductions(nu):
    th = theta(sigma1sq=1.7, c=13.0, a=2.5, gamma=0.6, alpha=0.7, delta=0.3, nu=nu)
    # correlation 1 at zero lag: C(0,0) = sigma1^2
    assert oracle.cov(th, 0.0, 0.0) == pytest.approx(1.7, rel=1e-15)
    # u = 0: isotropic Matern with decay c (Sect. 3, below Eq. (2))
    for h in [0.01, 0.1, 0.4]:
        assert oracle.cov(th, h, 0.0) == pytest.approx(1.7 * oracle.matern(nu, 13.0 * h), rel=1e-14)
    # h = 0: sigma1^2 (a|u|^{2 alpha} + 1)^{-(delta + gamma)}
    for u in [1.0, 2.0, 7.5]:
        assert oracle.cov(th, 0.0, u) == pytest.approx(1.7 * (2.5 * u ** 1.4 + 1) ** -(0.9), rel=1e-14)
    # gamma = 0: separable, C(h,u) C(0,0) = C(h,0) C(0,u)
    th0 = th.copy()
    th0[3] = 0.0
    for h, u in [(0.05, 1.0), (0.2, 3.0), (0.0, 2.0), (0.3, 0.0)]:
        assert oracle.cov(th0, h, u) * oracle.cov(th0, 0, 0) == pytest.approx(
            oracle.cov(th0, h, 0) * oracle.cov(th0, 0, u), rel=1e-14)
    # gamma > 0: NOT separable (the interaction of Eq. (2))
    assert abs(oracle.cov(th, 0.1, 2.0) * oracle.cov(th, 0, 0)
               - oracle.cov(th, 0.1, 0) * oracle.cov(th, 0, 2.0)) > 1e-4
    # symmetric in the sign of the lag
    assert oracle.cov(th, 0.1, -2.0) == oracle.cov(th, 0.1, 2.0)


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_cov_gradient_vs_central_differences(nu):
    th = theta(sigma1sq=1.3, c=20.0, a=3.0, gamma=0.45, alpha=0.4, delta=0.2, nu=nu)
    for h, u in [(0.03, 0.0), (0.07, 1.0), (0.15, 2.0), (0.0, 3.0), (0.01, 5.0)]:
        g = oracle.cov_grad(th, h, u)
        for p in range(4):
            e = 1e-6 * max(1.0, abs(th[p]))
            tp, tm = th.copy(), th.copy()
            tp[p] += e
            tm[p] -= e
            fd = (oracle.cov(tp, h, u) - oracle.cov(tm, h, u)) / (2 * e)
            assert g[p] == pytest.approx(fd, rel=1e-6, abs=1e-9), (h, u, p)


def test_theta_from_ranges_roundtrip():
    for (s, rs, rt, g, nug, al, de, nu) in [(1, 0.1, 3, 0.5, 0.05, 0.4, 0.2, 1.5),
                                            (2, 0.08, 5, 0.9, 0.1, 0.7, 0.1, 0.5),
                                            (1, 0.3, 1, 0.1, 0.2, 0.4, 0.2, 2.5)]:
        th = oracle.theta_from_ranges(s, rs, rt, g, nug, al, de, nu)
        assert oracle.cov(th, rs, 0.0) / s == pytest.approx(0.05, rel=1e-12)
        assert oracle.cov(th, 0.0, rt) / s == pytest.approx(0.05, rel=1e-12)
    # the spatial constant for nu = 1.5: (1 + x) e^{-x} = 0.05 at x = 4.7439 (4 decimals)
    th = oracle.theta_from_ranges(1, 1.0, 1, 0.5, 0.05, 0.4, 0.2, 1.5)
    assert round(th[1], 4) == 4.7439
    th = oracle.theta_from_ranges(1, 1.0, 1, 0.5, 0.05, 0.4, 0.2, 0.5)
    assert th[1] == pytest.approx(-math.log(0.05), rel=1e-12)
