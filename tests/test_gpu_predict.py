"""Vecchia prediction on the GPU (vecchia_predict) against the prediction
oracle: neighbour sets bit-exact (except near-ties, 1e-12 relative), mean and
variance within 1e-10 (FP64); the m = n case against exact kriging; edge
cases; sampled points at full size.

Mixed precision: the mean is first order in A_p, which the FP32 rounding of
the local covariance perturbs by up to cond(K_N) 2^-24 relative (rows with
cond > 1e4 are redone in FP64), so the mean is held to 1e-4 of the predictive
standard deviation and the variance (stationary in A_p) to 1e-5 relative."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import oracle.predict as opred
import synthetic_inputs as si
from gpu_util import cuda_or_skip, dev, load_vst

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return cuda_or_skip(), load_vst()


def pred_points(n, days, seed):
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.random((n, 2))), rng.integers(-1, days + 2, n).astype(float)


def check_mixed(mean, var, mean64, var64):
    sd = np.sqrt(var64)
    assert np.all(np.abs(mean - mean64) <= 1e-4 * sd)
    np.testing.assert_allclose(var, var64, rtol=1e-5)


def check_nn(nn_g, nn_o, xy, t, xyp, tp, th):
    R = oracle.cov_matrix(xyp, tp, xy, t, th) / th[0]
    for p in np.nonzero((nn_g != nn_o).any(1))[0]:
        # allowed only where the correlations of the differing entries tie
        a, b = nn_g[p], nn_o[p]
        ok = a >= 0
        assert np.all((a >= 0) == (b >= 0))
        ra, rb = R[p, a[ok]], R[p, b[ok]]
        assert np.allclose(ra, rb, rtol=1e-12, atol=0), p


@pytest.mark.parametrize("m", [10, 30])
def test_predict_parity(env, m):
    torch, vst = env
    w = si.tiny_uniform()
    th = oracle.theta_native(w.theta)
    xyp, tp = pred_points(300, 10, 5)
    # a few prediction points on top of training points
    xyp[:5], tp[:5] = w.xy[:5], w.t[:5]
    mo, vo, nno = opred.predict(w.xy, w.t, w.z, xyp, tp, th, m)
    _, vlo, _ = opred.predict(w.xy, w.t, w.z, xyp, tp, th, m, latent=True)
    xy_d, t_d, y_d, xyp_d, tp_d = dev(torch, w.xy, w.t, w.z, xyp, tp)
    mg, vg, nng = vst.vecchia_predict(xy_d, t_d, y_d, th, m, xyp_d, tp_d, precision=vst.FP64, nn=True)
    check_nn(nng.cpu().numpy(), nno, w.xy, w.t, xyp, tp, th)
    np.testing.assert_allclose(mg.cpu().numpy(), mo, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(vg.cpu().numpy(), vo, rtol=1e-10, atol=1e-10)
    _, vlg = vst.vecchia_predict(xy_d, t_d, y_d, th, m, xyp_d, tp_d, precision=vst.FP64, latent=True)
    np.testing.assert_allclose(vlg.cpu().numpy(), vlo, rtol=1e-10, atol=1e-10)
    mm, vm = vst.vecchia_predict(xy_d, t_d, y_d, th, m, xyp_d, tp_d, precision=vst.MIXED)
    check_mixed(mm.cpu().numpy(), vm.cpu().numpy(), mo, vo)


def test_predict_all_training_points_is_kriging(env):
    torch, vst = env
    st = si.stations_uniform(6, 4)
    xy, t = si.station_days(st, 4)                       # n = 24 <= VST_MAX_M
    th = oracle.theta_from_ranges(1.0, 0.3, 3.0, 0.5, 0.05)
    y = oracle.dense_sample(xy, t, th, si.standard_normal(t.shape[0], 2))
    xyp, tp = pred_points(40, 4, 9)
    n = t.shape[0]
    K = oracle.cov_matrix(xy, t, xy, t, th) + th[4] * np.eye(n)
    cf = sla.cho_factor(K, lower=True)
    Kp = oracle.cov_matrix(xy, t, xyp, tp, th)
    V = sla.solve_triangular(cf[0], Kp, lower=True)
    mean_ref, var_ref = Kp.T @ sla.cho_solve(cf, y), th[0] + th[4] - (V * V).sum(0)
    xy_d, t_d, y_d, xyp_d, tp_d = dev(torch, xy, t, y, xyp, tp)
    mg, vg = vst.vecchia_predict(xy_d, t_d, y_d, th, n, xyp_d, tp_d, precision=vst.FP64)
    np.testing.assert_allclose(mg.cpu().numpy(), mean_ref, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(vg.cpu().numpy(), var_ref, rtol=1e-9, atol=1e-10)


def test_predict_edge_cases(env):
    torch, vst = env
    w = si.tiny_uniform()
    th = oracle.theta_native(w.theta)
    xyp, tp = pred_points(50, 10, 7)
    xy_d, t_d, y_d, xyp_d, tp_d = dev(torch, w.xy, w.t, w.z, xyp, tp)
    # no training points: the prior
    mg, vg = vst.vecchia_predict(xy_d[:0], t_d[:0], y_d[:0], th, 10, xyp_d, tp_d)
    assert np.all(mg.cpu().numpy() == 0) and np.allclose(vg.cpu().numpy(), th[0] + th[4])
    # m = 0: the prior as well
    mg, vg = vst.vecchia_predict(xy_d, t_d, y_d, th, 0, xyp_d, tp_d)
    assert np.all(mg.cpu().numpy() == 0) and np.allclose(vg.cpu().numpy(), th[0] + th[4])
    # fewer training points than m
    mo, vo, _ = opred.predict(w.xy[:7], w.t[:7], w.z[:7], xyp, tp, th, 10)
    mg, vg = vst.vecchia_predict(xy_d[:7].contiguous(), t_d[:7].contiguous(), y_d[:7].contiguous(), th, 10, xyp_d,
                                 tp_d)
    np.testing.assert_allclose(mg.cpu().numpy(), mo, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(vg.cpu().numpy(), vo, rtol=1e-10, atol=1e-10)
    # no prediction points
    out = vst.vecchia_predict(xy_d, t_d, y_d, th, 10, xyp_d[:0], tp_d[:0])
    assert out[0].numel() == 0


def test_predict_fullsize_sampled(env):
    torch, vst = env
    w = si.continental()
    th = oracle.theta_native(w.theta)
    # next day at every station, plus off-network points
    last = w.t.max()
    st_xy = np.unique(w.xy[w.t == last], axis=0)
    rng = np.random.default_rng(3)
    off = st_xy[rng.choice(st_xy.shape[0], 200, replace=False)] + 0.01 * rng.standard_normal((200, 2))
    xyp = np.ascontiguousarray(np.concatenate([st_xy, off]))
    tp = np.full(xyp.shape[0], last + 1.0)
    xy_d, t_d, y_d, xyp_d, tp_d = dev(torch, w.xy, w.t, w.z, xyp, tp)
    mg, vg, nng = vst.vecchia_predict(xy_d, t_d, y_d, th, w.m, xyp_d, tp_d, precision=vst.MIXED, nn=True)
    m64, v64 = vst.vecchia_predict(xy_d, t_d, y_d, th, w.m, xyp_d, tp_d, precision=vst.FP64)
    mg, vg, nng, m64, v64 = (a.cpu().numpy() for a in (mg, vg, nng, m64, v64))
    check_mixed(mg, vg, m64, v64)
    sample = rng.choice(xyp.shape[0], 12, replace=False)
    mo, vo, nno = opred.predict(w.xy, w.t, w.z, xyp[sample], tp[sample], th, w.m)
    check_nn(nng[sample], nno, w.xy, w.t, xyp[sample], tp[sample], th)
    np.testing.assert_allclose(m64[sample], mo, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(v64[sample], vo, rtol=1e-10, atol=1e-10)
