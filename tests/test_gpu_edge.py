"""Edge cases of the CUDA path: empty and single-row inputs, m = 0 and the
maximum m, ragged first rows, non-integer and long time lags, duplicated
points, and device-side detection of invalid neighbour lists."""
import math

import numpy as np
import pytest

import oracle
import synthetic_inputs as si
from gpu_util import check_neighbours, cuda_or_skip, dev, load_vst

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = cuda_or_skip()
    return torch, load_vst()


def pts(n_st, n_days, seed, jitter=0.0, tscale=1.0):
    st = si.stations_uniform(n_st, seed)
    xy, t = si.station_days(st, n_days)
    t = t * tscale
    if jitter:
        t = t + jitter * np.random.default_rng(seed).random(t.shape[0])
    order = si.random_order(t.shape[0], seed)
    return np.ascontiguousarray(xy[order]), np.ascontiguousarray(t[order])


def roundtrip(torch, vst, xy, t, th, m, y, prec):
    xy_d, t_d, y_d = dev(torch, xy, t, y)
    nn, cnt, rm, rm1 = oracle.knn(xy, t, th, m)
    ws = vst.Workspace(t.shape[0], m)
    nn_g, cnt_g = vst.vif_build_neighbors(xy_d, t_d, th, m, ws=ws)
    vst.vst_workspace_status(ws)
    check_neighbours(nn_g.cpu().numpy(), cnt_g.cpu().numpy(), nn, cnt, rm, rm1)
    nn_d, cnt_d = dev(torch, nn, cnt)
    v, g = vst.vecchia_nll_grad(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=prec, ws=ws)
    vst.vst_workspace_status(ws)
    vo, go = oracle.nll_grad(xy, t, th, m, nn, cnt, y)
    return v.item(), g.cpu().numpy(), vo, go


def test_empty_and_single(env):
    torch, vst = env
    th = vst.vst_theta_from_ranges(1.0, 0.1, 3.0, 0.5, 0.05)
    for n in (0, 1):
        xy = np.random.default_rng(1).random((n, 2))
        t = np.zeros(n)
        y = np.full(n, 0.7)
        xy_d, t_d, y_d = dev(torch, xy, t, y)
        nn, cnt = vst.vif_build_neighbors(xy_d, t_d, th, 5)
        assert cnt.cpu().numpy().tolist() == [0] * n
        v, g = vst.vecchia_nll_grad(xy_d, t_d, th, 5, nn, cnt, y_d)
        s = th[0] + th[4]
        ref = 0.0 if n == 0 else 0.5 * math.log(2 * math.pi) + 0.5 * math.log(s) + 0.5 * 0.49 / s
        assert v.item() == pytest.approx(ref, abs=1e-14)


@pytest.mark.parametrize("m", [0, 1, 7, 15, 16, 31])
@pytest.mark.parametrize("prec", [0, 1])
def test_neighbour_counts(env, m, prec):
    torch, vst = env
    xy, t = pts(60, 6, 3)
    th = oracle.theta_from_ranges(1.0, 0.15, 2.0, 0.6, 0.08)
    y = si.standard_normal(t.shape[0], 4)
    v, g, vo, go = roundtrip(torch, vst, xy, t, th, m, y, prec)
    tol = 1e-10 if prec == 0 else 1e-6
    assert abs(v - vo) / t.shape[0] <= tol
    if prec == 0:
        np.testing.assert_allclose(g, go, rtol=1e-8, atol=1e-8 * np.abs(go).max())


def test_non_integer_and_long_lags(env):
    torch, vst = env
    # jittered times (no lag table) and a 5,000-day span (beyond the lag table)
    for jitter, tscale in ((0.37, 1.0), (0.0, 700.0), (0.5, 300.0)):
        xy, t = pts(50, 8, 5, jitter=jitter, tscale=tscale)
        th = oracle.theta_from_ranges(1.0, 0.2, 4.0 * tscale, 0.5, 0.05)
        y = si.standard_normal(t.shape[0], 6)
        for prec in (0, 1):
            v, g, vo, go = roundtrip(torch, vst, xy, t, th, 12, y, prec)
            assert abs(v - vo) / t.shape[0] <= (1e-10 if prec == 0 else 1e-6)


def test_duplicate_points(env):
    torch, vst = env
    xy, t = pts(30, 4, 7)
    xy = np.concatenate([xy, xy[:50]])
    t = np.concatenate([t, t[:50]])
    th = oracle.theta_from_ranges(1.0, 0.2, 3.0, 0.5, 0.1)
    y = si.standard_normal(t.shape[0], 8)
    v, g, vo, go = roundtrip(torch, vst, xy, t, th, 10, y, 0)
    assert abs(v - vo) / t.shape[0] <= 1e-10


def test_invalid_neighbour_list_is_reported(env):
    torch, vst = env
    xy, t = pts(20, 3, 9)
    th = oracle.theta_from_ranges(1.0, 0.2, 3.0, 0.5, 0.1)
    nn, cnt, _, _ = oracle.knn(xy, t, th, 5)
    nn[30, 2] = 40  # not a predecessor of row 30
    xy_d, t_d, y_d, nn_d, cnt_d = dev(torch, xy, t, si.standard_normal(t.shape[0], 1), nn, cnt)
    ws = vst.Workspace(t.shape[0], 5)
    vst.vecchia_nll(xy_d, t_d, th, 5, nn_d, cnt_d, y_d, ws=ws)
    with pytest.raises(vst.VstError) as e:
        vst.vst_workspace_status(ws)
    assert e.value.code == 1 and e.value.info["bad_row"] == 30
    # the workspace is usable again afterwards
    nn[30, 2] = 3
    nn_d = dev(torch, nn)[0]
    vst.vecchia_nll(xy_d, t_d, th, 5, nn_d, cnt_d, y_d, ws=ws)
    assert vst.vst_workspace_status(ws)["status"] == 0
