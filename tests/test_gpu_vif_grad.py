"""VIF gradient (Sect. 4.3 likelihood, FP64 and mixed) on the GPU against the
forward-mode oracle of oracle/vif.py, on the oracle's neighbour sets.

Tolerance: both sides are FP64; the reverse-mode GPU path and the forward-mode
oracle take different routes through Sigma_kk^{-1} and M^{-1}, whose
condition numbers (<= ~1e6 for these kMeans++ inducing sets) amplify the
2^-53 rounding, and the gradient is a sum of n terms of size O(1): so
|dg_j| <= 1e-7 |g_j| + 1e-9 n."""
import numpy as np
import pytest

import oracle
import oracle.vif as ovif
import synthetic_inputs as si
from gpu_util import cuda_or_skip, dev, load_vst

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


def check(g, g_o, n):
    g, g_o = np.asarray(g), np.asarray(g_o)
    err = np.abs(g - g_o)
    assert np.all(err <= 1e-7 * np.abs(g_o) + 1e-9 * n), (g, g_o, err)


# cases: several 64-wide column tiles of the dense k-products with a ragged
# tail (k = 70, 130), more than one 1024-row block of the reverse-index scan
# (n = 1200), k = 1, random and time orderings, m = 0 (FITC)
@pytest.mark.parametrize("n_st,n_days,k,m,order", [
    (40, 10, 24, 8, "time"),
    (30, 12, 70, 12, "random"),
    (60, 20, 130, 6, "time"),
    (30, 8, 1, 5, "time"),
    (30, 8, 20, 0, "random"),
])
def test_vif_grad_parity(env, n_st, n_days, k, m, order):
    torch, vst = env
    xy, t, th, xyk, tk, y = problem(n_st, n_days, k, seed=k + m + n_days, order=order)
    n = t.shape[0]
    U, r = ovif.lowrank(xy, t, xyk, tk, th)
    if m > 0:
        nn, cnt, _, _ = ovif.knn(xy, t, th, U, r, m)
    else:
        nn = np.zeros((n, 0), dtype=np.int32)
        cnt = np.zeros(n, dtype=np.int32)
    v_o, g_o = ovif.nll_grad(xy, t, th, xyk, tk, m, nn, cnt, y)
    xy_d, t_d, y_d, xyk_d, tk_d, nn_d, cnt_d = dev(torch, xy, t, y, xyk, tk, nn, cnt)
    ind = (xyk_d, tk_d)
    nll, grad = vst.vecchia_nll_grad(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=vst.FP64, inducing=ind)
    torch.cuda.synchronize()
    assert abs(nll.item() - v_o) / n <= 1e-10
    check(grad.cpu().numpy(), g_o, n)
    # the NLL it returns is the FP64 VIF NLL, bit for bit
    v = vst.vecchia_nll(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=vst.FP64, inducing=ind)
    assert v.item() == nll.item()
    # repeated calls give the same bits (fixed-order reductions, sorted reverse index)
    nll2, grad2 = vst.vecchia_nll_grad(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=vst.FP64, inducing=ind)
    assert nll2.item() == nll.item() and torch.equal(grad2, grad)


def test_vif_grad_all_predecessors_is_exact_gp_gradient(env):
    # m = n-1: the exact GP gradient for any inducing set
    torch, vst = env
    xy, t, th, xyk, tk, y = problem(8, 4, 9, seed=5)  # n = 32, m = 31
    n = t.shape[0]
    m, nn, cnt = oracle.all_predecessors(n)
    assert m <= vst.MAX_M
    v0, g0 = oracle.dense_nll(xy, t, th, y, grad=True)
    xy_d, t_d, y_d, xyk_d, tk_d, nn_d, cnt_d = dev(torch, xy, t, y, xyk, tk, nn, cnt)
    nll, grad = vst.vecchia_nll_grad(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=vst.FP64,
                                     inducing=(xyk_d, tk_d))
    assert abs(nll.item() - v0) / n <= 1e-10
    check(grad.cpu().numpy(), g0, n)


# mixed forms: FP32 low rank, W and residual Gram from the tensor-core NLL,
# the dense products on the split-BF16 tensor cores, FP64 n-long reductions.
# The mixed NLL meets |dNLL| / n <= 1e-6; each of the n terms of a gradient
# component carries errors of the same FP32 origin, so the bar is
# |dg_j| <= 1e-6 n (+ 1e-4 |g_j|); observed <= 7e-8 n on these cases.
@pytest.mark.parametrize("precision", ["MIXED", "MIXED_BF16X3"])
@pytest.mark.parametrize("n_st,n_days,k,m,order", [
    (40, 10, 24, 8, "time"),
    (30, 12, 70, 12, "random"),
    (30, 8, 20, 0, "random"),
])
def test_vif_grad_mixed_parity(env, precision, n_st, n_days, k, m, order):
    torch, vst = env
    prec = getattr(vst, precision)
    xy, t, th, xyk, tk, y = problem(n_st, n_days, k, seed=k + m + n_days, order=order)
    n = t.shape[0]
    U, r = ovif.lowrank(xy, t, xyk, tk, th)
    if m > 0:
        nn, cnt, _, _ = ovif.knn(xy, t, th, U, r, m)
    else:
        nn = np.zeros((n, 0), dtype=np.int32)
        cnt = np.zeros(n, dtype=np.int32)
    v_o, g_o = ovif.nll_grad(xy, t, th, xyk, tk, m, nn, cnt, y)
    xy_d, t_d, y_d, xyk_d, tk_d, nn_d, cnt_d = dev(torch, xy, t, y, xyk, tk, nn, cnt)
    ind = (xyk_d, tk_d)
    nll, grad = vst.vecchia_nll_grad(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=prec, inducing=ind)
    assert abs(nll.item() - v_o) / n <= 1e-6
    err = np.abs(grad.cpu().numpy() - g_o)
    assert np.all(err <= 1e-4 * np.abs(g_o) + 1e-6 * n), (grad.cpu().numpy(), g_o, err)
    # the NLL it returns is the mixed VIF NLL of the same precision, bit for bit
    v = vst.vecchia_nll(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=prec, inducing=ind)
    assert v.item() == nll.item()


def test_vif_grad_small_workspace(env):
    torch, vst = env
    xy, t, th, xyk, tk, y = problem(10, 4, 8, seed=2)
    n = t.shape[0]
    U, r = ovif.lowrank(xy, t, xyk, tk, th)
    nn, cnt, _, _ = ovif.knn(xy, t, th, U, r, 4)
    xy_d, t_d, y_d, xyk_d, tk_d, nn_d, cnt_d = dev(torch, xy, t, y, xyk, tk, nn, cnt)
    ws = vst.Workspace(n, 4, 8)  # the NLL's workspace: too small for the gradient
    with pytest.raises(ValueError):
        vst.vecchia_nll_grad(xy_d, t_d, th, 4, nn_d, cnt_d, y_d, precision=vst.FP64, inducing=(xyk_d, tk_d), ws=ws)


@pytest.mark.parametrize("n", [0, 1, 5])
@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
def test_vif_grad_empty_and_tiny(env, n, precision):
    """n = 0 (NLL and gradient 0), a single point, and n <= m (every row's
    neighbours are all its predecessors), with k = 3 inducing points."""
    torch, vst = env
    prec = getattr(vst, precision)
    xy0, t0, th, xyk, tk, y0 = problem(10, 4, 3, seed=6)
    xy, t, y = (np.ascontiguousarray(a[:n]) for a in (xy0, t0, y0))
    m = 4
    xy_d, t_d, y_d, xyk_d, tk_d = dev(torch, xy, t, y, xyk, tk)
    ind = (xyk_d, tk_d)
    nn_d, cnt_d = vst.vif_build_neighbors(xy_d, t_d, th, m, inducing=ind)
    cnt = cnt_d.cpu().numpy()
    assert cnt.tolist() == [min(i, m) for i in range(n)]
    nll, grad = vst.vecchia_nll_grad(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=prec, inducing=ind)
    if n == 0:
        assert nll.item() == 0.0 and np.all(grad.cpu().numpy() == 0.0)
        return
    nn = nn_d.cpu().numpy()
    v_o, g_o = ovif.nll_grad(xy, t, th, xyk, tk, m, nn, cnt, y)
    tol_v, tol_g = (1e-10, 1e-7) if precision == "FP64" else (1e-6, 1e-4)
    assert abs(nll.item() - v_o) / n <= tol_v
    err = np.abs(grad.cpu().numpy() - g_o)
    assert np.all(err <= tol_g * np.abs(g_o) + 1e-6 * n), (grad.cpu().numpy(), g_o)
