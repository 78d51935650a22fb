"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: neighbour sets bit-exact except listed cut-off ties (< 1e-12
relative); FP64: |dNLL|/n <= 1e-10, A and D to 1e-9 absolute / relative,
gradient to 1e-8 relative; mixed precision: |dNLL|/n <= 1e-6 and, per
gradient component, |dg_j| <= 1e-4 |g_j| + 1e-6 n (the NLL's per-point bar
carried to each n-term sum of the gradient, plus a relative part)."""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si
from gpu_util import check_neighbours, cuda_or_skip, dev, load_vst

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def vst(torch):
    return load_vst()


def problem(w, nu=1.5):
    th = oracle.theta_from_ranges(*w.theta.astuple()[:5], w.theta.alpha, w.theta.delta, nu)
    return th


@pytest.fixture(scope="module")
def tiny(torch, vst):
    w = si.tiny_uniform(m=10)
    th = problem(w)
    nn, cnt, rm, rm1 = oracle.knn(w.xy, w.t, th, w.m)
    y = oracle.dense_sample(w.xy, w.t, th, w.z)
    xy_d, t_d, y_d = dev(torch, w.xy, w.t, y)
    return dict(w=w, th=th, nn=nn, cnt=cnt, rm=rm, rm1=rm1, y=y, xy=xy_d, t=t_d, yd=y_d)


def test_knn_tiny(tiny, vst, torch):
    w = tiny["w"]
    tie = torch.zeros(w.n, dtype=torch.int64, device="cuda")
    ws = vst.Workspace(w.n, w.m)
    nn_g, cnt_g = vst.vif_build_neighbors(tiny["xy"], tiny["t"], tiny["th"], w.m, tie_rows=tie, ws=ws)
    info = vst.vst_workspace_status(ws)
    ties = check_neighbours(nn_g.cpu().numpy(), cnt_g.cpu().numpy(), tiny["nn"], tiny["cnt"], tiny["rm"],
                            tiny["rm1"])
    # the GPU lists exactly the rows the oracle finds tied at the cut-off
    assert info["n_tie"] == len(ties)
    gt = sorted(tie.cpu().numpy()[:info["n_tie"]].tolist())
    assert gt == ties


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_fp64_factor_nll_grad_tiny(tiny, vst, torch, nu):
    w = tiny["w"]
    th = problem(w, nu)
    nn, cnt, _, _ = oracle.knn(w.xy, w.t, th, w.m)
    nn_d, cnt_d = dev(torch, nn, cnt)
    A, D = vst.vecchia_factor(tiny["xy"], tiny["t"], th, w.m, nn_d, cnt_d, precision=vst.FP64)
    A_o, D_o = oracle.factor(w.xy, w.t, th, w.m, nn, cnt)
    np.testing.assert_allclose(A.cpu().numpy(), A_o, atol=1e-9, rtol=0)
    np.testing.assert_allclose(D.cpu().numpy(), D_o, rtol=1e-9)
    v, g = vst.vecchia_nll_grad(tiny["xy"], tiny["t"], th, w.m, nn_d, cnt_d, tiny["yd"], precision=vst.FP64)
    v1 = vst.vecchia_nll(tiny["xy"], tiny["t"], th, w.m, nn_d, cnt_d, tiny["yd"], precision=vst.FP64)
    vo, go = oracle.nll_grad(w.xy, w.t, th, w.m, nn, cnt, tiny["y"])
    assert abs(v.item() - vo) / w.n <= 1e-10
    assert abs(v1.item() - vo) / w.n <= 1e-10
    np.testing.assert_allclose(g.cpu().numpy(), go, rtol=1e-8, atol=1e-8 * np.abs(go).max())


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_mixed_nll_grad_tiny(tiny, vst, torch, nu):
    w = tiny["w"]
    th = problem(w, nu)
    nn, cnt, _, _ = oracle.knn(w.xy, w.t, th, w.m)
    nn_d, cnt_d = dev(torch, nn, cnt)
    ws = vst.Workspace(w.n, w.m)
    v, g = vst.vecchia_nll_grad(tiny["xy"], tiny["t"], th, w.m, nn_d, cnt_d, tiny["yd"], precision=vst.MIXED, ws=ws)
    vst.vst_workspace_status(ws)
    vo, go = oracle.nll_grad(w.xy, w.t, th, w.m, nn, cnt, tiny["y"])
    assert abs(v.item() - vo) / w.n <= 1e-6
    assert np.all(np.abs(g.cpu().numpy() - go) <= 1e-4 * np.abs(go) + 1e-6 * w.n)
    A, D = vst.vecchia_factor(tiny["xy"], tiny["t"], th, w.m, nn_d, cnt_d, precision=vst.MIXED)
    A_o, D_o = oracle.factor(w.xy, w.t, th, w.m, nn, cnt)
    np.testing.assert_allclose(D.cpu().numpy(), D_o, rtol=1e-5)
    np.testing.assert_allclose(A.cpu().numpy(), A_o, atol=1e-4)


def test_gradient_central_differences_fp64(tiny, vst, torch):
    w = tiny["w"]
    th = np.array(tiny["th"])
    nn_d, cnt_d = dev(torch, tiny["nn"], tiny["cnt"])
    _, g = vst.vecchia_nll_grad(tiny["xy"], tiny["t"], th, w.m, nn_d, cnt_d, tiny["yd"])
    g = g.cpu().numpy()
    for p in range(5):
        e = 1e-6 * max(1.0, abs(th[p]))
        tp, tm = th.copy(), th.copy()
        tp[p] += e
        tm[p] -= e
        fp = vst.vecchia_nll(tiny["xy"], tiny["t"], tp, w.m, nn_d, cnt_d, tiny["yd"]).item()
        fm = vst.vecchia_nll(tiny["xy"], tiny["t"], tm, w.m, nn_d, cnt_d, tiny["yd"]).item()
        assert g[p] == pytest.approx((fp - fm) / (2 * e), rel=1e-5, abs=1e-4)


def test_sampling_and_whitening(tiny, vst, torch):
    w = tiny["w"]
    th = tiny["th"]
    nn, cnt = tiny["nn"], tiny["cnt"]
    nn_d, cnt_d, z_d = dev(torch, nn, cnt, w.z)
    ws = vst.Workspace(w.n, w.m)
    y = vst.vecchia_sample(tiny["xy"], tiny["t"], th, w.m, nn_d, cnt_d, z_d, ws=ws)
    vst.vst_workspace_status(ws)
    A_o, D_o = oracle.factor(w.xy, w.t, th, w.m, nn, cnt)
    y_o = oracle.vecchia_sample(w.m, nn, cnt, A_o, D_o, w.z)
    np.testing.assert_allclose(y.cpu().numpy(), y_o, atol=1e-9, rtol=1e-9)
    v = vst.vecchia_nll(tiny["xy"], tiny["t"], th, w.m, nn_d, cnt_d, y).item()
    ref = 0.5 * w.n * np.log(2 * np.pi) + 0.5 * np.log(D_o).sum() + 0.5 * (w.z ** 2).sum()
    assert abs(v - ref) / w.n <= 1e-10


def test_deterministic(tiny, vst, torch):
    w = tiny["w"]
    nn_d, cnt_d = dev(torch, tiny["nn"], tiny["cnt"])
    for prec in (vst.FP64, vst.MIXED):
        a = vst.vecchia_nll_grad(tiny["xy"], tiny["t"], tiny["th"], w.m, nn_d, cnt_d, tiny["yd"], precision=prec)
        b = vst.vecchia_nll_grad(tiny["xy"], tiny["t"], tiny["th"], w.m, nn_d, cnt_d, tiny["yd"], precision=prec)
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


@pytest.fixture(scope="module")
def box(torch, vst):
    w = si.box_uniform(m=20, n_days=20)  # 20,000 points: full oracle neighbour search stays quick
    th = problem(w)
    nn, cnt, rm, rm1 = oracle.knn(w.xy, w.t, th, w.m)
    A, D = oracle.factor(w.xy, w.t, th, w.m, nn, cnt)
    y = oracle.vecchia_sample(w.m, nn, cnt, A, D, w.z)
    xy_d, t_d, y_d = dev(torch, w.xy, w.t, y)
    return dict(w=w, th=th, nn=nn, cnt=cnt, rm=rm, rm1=rm1, A=A, D=D, y=y, xy=xy_d, t=t_d, yd=y_d)


def test_box_uniform_20k(box, vst, torch):
    w, th = box["w"], box["th"]
    ws = vst.Workspace(w.n, w.m)
    nn_g, cnt_g = vst.vif_build_neighbors(box["xy"], box["t"], th, w.m, ws=ws)
    vst.vst_workspace_status(ws)
    check_neighbours(nn_g.cpu().numpy(), cnt_g.cpu().numpy(), box["nn"], box["cnt"], box["rm"], box["rm1"])
    nn_d, cnt_d = dev(torch, box["nn"], box["cnt"])
    vo, go, gt = oracle.nll_grad(w.xy, w.t, th, w.m, box["nn"], box["cnt"], box["y"], terms=True)
    v64, g64 = vst.vecchia_nll_grad(box["xy"], box["t"], th, w.m, nn_d, cnt_d, box["yd"], precision=vst.FP64, ws=ws)
    assert abs(v64.item() - vo) / w.n <= 1e-10
    np.testing.assert_allclose(g64.cpu().numpy(), go, rtol=1e-8, atol=1e-9 * np.abs(gt).sum(0).max())
    vmx, gmx = vst.vecchia_nll_grad(box["xy"], box["t"], th, w.m, nn_d, cnt_d, box["yd"], precision=vst.MIXED, ws=ws)
    info = vst.vst_workspace_status(ws)
    assert abs(vmx.item() - vo) / w.n <= 1e-6
    assert np.all(np.abs(gmx.cpu().numpy() - go) <= 1e-4 * np.abs(go) + 1e-6 * w.n)
    # whitening identity with the oracle's factor
    ref = 0.5 * w.n * np.log(2 * np.pi) + 0.5 * np.log(box["D"]).sum() + 0.5 * (w.z ** 2).sum()
    assert abs(v64.item() - ref) / w.n <= 1e-10
    assert info["n_fallback"] == 0
