"""VIF (Sect. 4.3) on the GPU against the VIF oracle: residual-correlation
neighbour sets (bit-exact except listed cut-off ties, 1e-12 relative), the
residual factor (FP64: 1e-9), the Woodbury NLL (FP64: |dNLL|/n <= 1e-10;
mixed: <= 1e-6), the FITC special case m = 0 and k = 1."""
import numpy as np
import pytest

import oracle
import oracle.vif as ovif
import synthetic_inputs as si
from gpu_util import check_neighbours, cuda_or_skip, dev, load_vst

pytestmark = pytest.mark.gpu


def problem(n_st, n_days, k, seed, order="time", rs=0.12, rt=2.0, nug=0.05):
    st = si.stations_uniform(n_st, seed)
    xy, t = si.station_days(st, n_days)
    perm = si.time_stratified_order(t, seed) if order == "time" else si.random_order(t.shape[0], seed)
    xy, t = np.ascontiguousarray(xy[perm]), np.ascontiguousarray(t[perm])
    th = oracle.theta_from_ranges(1.0, rs, rt, 0.5, nug)
    X = np.concatenate([xy / rs, (t / rt)[:, None]], axis=1)
    C = si.kmeanspp(X, k, seed + 3, lloyd_iters=10)
    xyk, tk = np.ascontiguousarray(C[:, :2] * rs), np.ascontiguousarray(C[:, 2] * rt)
    y = oracle.dense_sample(xy, t, th, si.standard_normal(t.shape[0], seed + 9))
    return xy, t, th, xyk, tk, y


@pytest.fixture(scope="module")
def env():
    return cuda_or_skip(), load_vst()


@pytest.mark.parametrize("k,m,order", [(24, 8, "time"), (40, 12, "random"), (1, 5, "time")])
def test_vif_neighbours_factor_nll(env, k, m, order):
    torch, vst = env
    xy, t, th, xyk, tk, y = problem(40, 10, k, seed=k + m, order=order)
    n = t.shape[0]
    U, r = ovif.lowrank(xy, t, xyk, tk, th)
    nn_o, cnt_o, rm, rm1 = ovif.knn(xy, t, th, U, r, m)
    xy_d, t_d, y_d, xyk_d, tk_d = dev(torch, xy, t, y, xyk, tk)
    ind = (xyk_d, tk_d)
    ws = vst.Workspace(n, m, k)
    nn_g, cnt_g = vst.vif_build_neighbors(xy_d, t_d, th, m, ws=ws, inducing=ind)
    vst.vst_workspace_status(ws)
    check_neighbours(nn_g.cpu().numpy(), cnt_g.cpu().numpy(), nn_o, cnt_o, rm, rm1)
    nn_d, cnt_d = dev(torch, nn_o, cnt_o)
    A_o, D_o = ovif.factor(xy, t, th, U, m, nn_o, cnt_o)
    A, D = vst.vecchia_factor(xy_d, t_d, th, m, nn_d, cnt_d, precision=vst.FP64, ws=ws, inducing=ind)
    vst.vst_workspace_status(ws)
    np.testing.assert_allclose(A.cpu().numpy(), A_o, atol=1e-9)
    np.testing.assert_allclose(D.cpu().numpy(), D_o, rtol=1e-9)
    v_o = ovif.nll(xy, t, th, U, m, nn_o, cnt_o, y, A_o, D_o)
    v = vst.vecchia_nll(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=vst.FP64, ws=ws, inducing=ind)
    vst.vst_workspace_status(ws)
    assert abs(v.item() - v_o) / n <= 1e-10
    vm = vst.vecchia_nll(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=vst.MIXED, ws=ws, inducing=ind)
    vst.vst_workspace_status(ws)
    assert abs(vm.item() - v_o) / n <= 1e-6


def test_vif_neighbours_short_range_uses_brute_force_rows(env):
    """Residual correlations all tiny (effective ranges far below the point
    spacing): the FP32 filter cannot separate them, every predecessor stays
    a candidate, rows past the candidate capacity (256) are searched by the
    FP64 brute force and the rest ranked from their full candidate lists."""
    torch, vst = env
    xy, t, th, xyk, tk, y = problem(40, 8, 16, seed=3, rs=0.01, rt=0.05)
    n = t.shape[0]
    assert n > 300
    m = 6
    U, r = ovif.lowrank(xy, t, xyk, tk, th)
    nn_o, cnt_o, rm, rm1 = ovif.knn(xy, t, th, U, r, m)
    xy_d, t_d, xyk_d, tk_d = dev(torch, xy, t, xyk, tk)
    ws = vst.Workspace(n, m, 16)
    nn_g, cnt_g = vst.vif_build_neighbors(xy_d, t_d, th, m, ws=ws, inducing=(xyk_d, tk_d))
    vst.vst_workspace_status(ws)
    check_neighbours(nn_g.cpu().numpy(), cnt_g.cpu().numpy(), nn_o, cnt_o, rm, rm1)


def test_vif_neighbours_non_integer_times(env):
    """Times that are not whole days: the FP32 tile filter cannot bound the
    lag rounding and keeps every pair of such tiles (rows beyond the
    candidate capacity go through the second pass, which evaluates those
    lags exactly in FP64)."""
    torch, vst = env
    xy, t, th, xyk, tk, y = problem(40, 8, 20, seed=8, order="random")
    t = np.ascontiguousarray(t + 0.37 * si.stations_uniform(t.shape[0], 21)[:, 0])
    n = t.shape[0]
    m = 7
    U, r = ovif.lowrank(xy, t, xyk, tk, th)
    nn_o, cnt_o, rm, rm1 = ovif.knn(xy, t, th, U, r, m)
    xy_d, t_d, xyk_d, tk_d = dev(torch, xy, t, xyk, tk)
    ws = vst.Workspace(n, m, 20)
    nn_g, cnt_g = vst.vif_build_neighbors(xy_d, t_d, th, m, ws=ws, inducing=(xyk_d, tk_d))
    vst.vst_workspace_status(ws)
    check_neighbours(nn_g.cpu().numpy(), cnt_g.cpu().numpy(), nn_o, cnt_o, rm, rm1)


def test_vif_m0_is_fitc(env):
    torch, vst = env
    xy, t, th, xyk, tk, y = problem(30, 6, 16, seed=4)
    n = t.shape[0]
    U, r = ovif.lowrank(xy, t, xyk, tk, th)
    nn = np.zeros((n, 0), dtype=np.int32)
    cnt = np.zeros(n, dtype=np.int32)
    v_o = ovif.nll(xy, t, th, U, 0, nn, cnt, y)
    xy_d, t_d, y_d, xyk_d, tk_d, nn_d, cnt_d = dev(torch, xy, t, y, xyk, tk, nn, cnt)
    v = vst.vecchia_nll(xy_d, t_d, th, 0, nn_d, cnt_d, y_d, precision=vst.FP64, inducing=(xyk_d, tk_d))
    assert abs(v.item() - v_o) / n <= 1e-10


@pytest.mark.parametrize("n_st,n_days,k", [(40, 8, 24), (60, 5, 257), (30, 12, 300)])
def test_lowrank_u_parity(env, n_st, n_days, k):
    """U = Sigma_nk L^{-T} and r = sigma1^2 - ||U_i||^2 against the oracle:
    the FP64 GEMM, and the tensor-core GEMM with six and with three
    split-BF16 products.  Cases span several 128-row tiles with a ragged tail,
    k padded to the 256-wide tiles, and k % 4 != 0 (scalar stores).
    Tolerances, relative to max |U| (r: to sigma1^2): FP64 1e-12; six
    products 1e-5 (FP32 covariance entries, about 1e-7 relative, amplified by
    the large entries of L^{-1} when k is close to n); three products 1e-4
    (16 significand bits per operand, ~1e-5 per entry)."""
    torch, vst = env
    xy, t, th, xyk, tk, _ = problem(n_st, n_days, k, seed=k, order="random")
    U_o, r_o = ovif.lowrank(xy, t, xyk, tk, th)
    xy_d, t_d, xyk_d, tk_d = dev(torch, xy, t, xyk, tk)
    scale = np.abs(U_o).max()
    for prec, tol in ((vst.FP64, 1e-12), (vst.MIXED, 1e-5), (vst.MIXED_BF16X3, 1e-4)):
        ws = vst.Workspace(t.shape[0], 0, k)
        U, r = vst.vif_lowrank_u(xy_d, t_d, th, (xyk_d, tk_d), precision=prec, ws=ws)
        vst.vst_workspace_status(ws)
        assert np.abs(U.cpu().numpy() - U_o).max() <= tol * scale, prec
        assert np.abs(r.cpu().numpy() - r_o).max() <= tol * th[0], prec


def test_vif_nll_split_bf16_forms(env):
    """VIF NLL with the tensor-core low rank, both split forms, against the
    oracle's Woodbury NLL: |dNLL|/n <= 1e-6 (six products) and <= 1e-5
    (three products)."""
    torch, vst = env
    k, m = 60, 10
    xy, t, th, xyk, tk, y = problem(40, 10, k, seed=17, order="time")
    n = t.shape[0]
    U, r = ovif.lowrank(xy, t, xyk, tk, th)
    nn_o, cnt_o, _, _ = ovif.knn(xy, t, th, U, r, m)
    v_o = ovif.nll(xy, t, th, U, m, nn_o, cnt_o, y)
    xy_d, t_d, y_d, xyk_d, tk_d, nn_d, cnt_d = dev(torch, xy, t, y, xyk, tk, nn_o, cnt_o)
    ws = vst.Workspace(n, m, k)
    for prec, tol in ((vst.MIXED, 1e-6), (vst.MIXED_BF16X3, 1e-5)):
        v = vst.vecchia_nll(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=prec, ws=ws, inducing=(xyk_d, tk_d))
        vst.vst_workspace_status(ws)
        assert abs(v.item() - v_o) / n <= tol, (prec, abs(v.item() - v_o) / n)


def test_vif_grad_tensor_core_gram_many_drains(env):
    """n = 20,000, k = 40: the mixed gradient's J = H^T U on the split-K
    tensor-core Gram, where each CTA drains its two tensor-memory buffers ~10
    times, against the FP64 gradient (which the oracle pins at small n):
    |dg_j| <= 1e-4 |g_j| + 1e-6 n.  The mixed NLL of both split forms against
    the oracle's Woodbury NLL, |dNLL|/n <= 1e-6.  Conditioning sets: the m
    previous points (any predecessor sets define a Vecchia NLL); responses
    standard normal."""
    torch, vst = env
    k, m = 40, 8
    st = si.stations_uniform(200, 23)
    xy, t = si.station_days(st, 100)
    perm = si.time_stratified_order(t, 23)
    xy, t = np.ascontiguousarray(xy[perm]), np.ascontiguousarray(t[perm])
    n = t.shape[0]
    th = oracle.theta_from_ranges(1.0, 0.12, 2.0, 0.5, 0.05)
    X = np.concatenate([xy / 0.12, (t / 2.0)[:, None]], axis=1)
    C = si.kmeanspp(X, k, 26, lloyd_iters=5)
    xyk, tk = np.ascontiguousarray(C[:, :2] * 0.12), np.ascontiguousarray(C[:, 2] * 2.0)
    y = si.standard_normal(n, 29)
    cnt = np.minimum(np.arange(n), m).astype(np.int32)
    nn = np.zeros((n, m), dtype=np.int32)
    for j in range(m):
        nn[:, j] = np.maximum(np.arange(n) - 1 - j, 0)
    U, _ = ovif.lowrank(xy, t, xyk, tk, th)
    v_o = ovif.nll(xy, t, th, U, m, nn, cnt, y)
    xy_d, t_d, y_d, xyk_d, tk_d, nn_d, cnt_d = dev(torch, xy, t, y, xyk, tk, nn, cnt)
    ind = (xyk_d, tk_d)
    ws = vst.Workspace(n, m, k, vif_grad=True)
    for prec in (vst.MIXED, vst.MIXED_BF16X3):
        v = vst.vecchia_nll(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=prec, ws=ws, inducing=ind)
        vst.vst_workspace_status(ws)
        print("dNLL/n", prec, abs(v.item() - v_o) / n)
        assert abs(v.item() - v_o) / n <= 1e-6, (prec, abs(v.item() - v_o) / n)
    _, g64 = vst.vecchia_nll_grad(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=vst.FP64, ws=ws, inducing=ind)
    _, gm = vst.vecchia_nll_grad(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=vst.MIXED, ws=ws, inducing=ind)
    vst.vst_workspace_status(ws)
    g64, gm = g64.cpu().numpy(), gm.cpu().numpy()
    print("grad mixed - fp64 per n", (gm - g64) / n)
    assert np.all(np.abs(gm - g64) <= 1e-4 * np.abs(g64) + 1e-6 * n), (gm, g64)


@pytest.mark.parametrize("k,m", [(60, 30), (130, 26), (61, 31)])
def test_vif_mixed_32_position_blocks(env, k, m):
    """Local blocks of 32 positions (m = 24..31), whose per-row residual Gram
    runs on the tensor cores (groups of four rows, 64-column chunks; here
    410 rows: the last group ragged, for k = 130 a ragged last chunk, for
    k = 61 an odd column count, and m = 31 a block without padding):
    the mixed NLL and NLL + gradient against the oracle's Woodbury NLL and
    forward-mode gradient, |dNLL|/n <= 1e-6, |dg_j| <= 1e-4 |g_j| + 1e-6 n."""
    torch, vst = env
    xy, t, th, xyk, tk, y = problem(41, 10, k, seed=k + m, order="time")
    n = t.shape[0]
    U, r = ovif.lowrank(xy, t, xyk, tk, th)
    nn_o, cnt_o, _, _ = ovif.knn(xy, t, th, U, r, m)
    v_o, g_o = ovif.nll_grad(xy, t, th, xyk, tk, m, nn_o, cnt_o, y)
    xy_d, t_d, y_d, xyk_d, tk_d, nn_d, cnt_d = dev(torch, xy, t, y, xyk, tk, nn_o, cnt_o)
    ind = (xyk_d, tk_d)
    ws = vst.Workspace(n, m, k, vif_grad=True)
    for prec in (vst.MIXED, vst.MIXED_BF16X3):
        v = vst.vecchia_nll(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=prec, ws=ws, inducing=ind)
        vst.vst_workspace_status(ws)
        assert abs(v.item() - v_o) / n <= 1e-6, (prec, abs(v.item() - v_o) / n)
        v2, g = vst.vecchia_nll_grad(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=prec, ws=ws, inducing=ind)
        vst.vst_workspace_status(ws)
        assert v2.item() == v.item()
        err = np.abs(g.cpu().numpy() - g_o)
        assert np.all(err <= 1e-4 * np.abs(g_o) + 1e-6 * n), (prec, g.cpu().numpy(), g_o)
