"""vecchia_nll_grad_noalloc against vecchia_nll_grad.

The no-allocation entry point serves callers that cannot call cudaMalloc
(a host application that owns every device allocation, or a latency-critical
path that cannot take cudaMalloc's implicit synchronisation); it takes its
scratch from the library's static device array instead of a workspace.  Its
results must be those of the workspace-based entry point, call after call
(the array keeps the previous call's contents and must be reset correctly).
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run alone."""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si
from gpu_util import cuda_or_skip, dev, load_vst

pytestmark = pytest.mark.gpu


def test_noalloc_matches_workspace_entry_point():
    torch = cuda_or_skip()
    vst = load_vst()
    w = si.tiny_uniform(m=10)
    th = oracle.theta_native(w.theta)
    nn, cnt, _, _ = oracle.knn(w.xy, w.t, th, w.m)
    y = oracle.dense_sample(w.xy, w.t, th, w.z)
    xy_d, t_d, y_d, nn_d, cnt_d = dev(torch, w.xy, w.t, y, nn, cnt)
    for prec in (vst.FP64, vst.MIXED):
        ws = vst.Workspace(w.n, w.m)
        v_ref, g_ref = vst.vecchia_nll_grad(xy_d, t_d, th, w.m, nn_d, cnt_d, y_d, precision=prec, ws=ws)
        vst.vst_workspace_status(ws)
        v_ref, g_ref = v_ref.item(), g_ref.cpu().numpy()
        nll = torch.empty(1, dtype=torch.float64, device="cuda")
        grad = torch.empty(5, dtype=torch.float64, device="cuda")
        for call in range(2):  # two calls in a row share the static scratch
            nll.fill_(np.nan)
            grad.fill_(np.nan)
            vst.vecchia_nll_grad_noalloc(xy_d, t_d, th, w.m, nn_d, cnt_d, y_d, precision=prec, nll=nll, grad=grad)
            info = vst.vst_noalloc_status()
            assert info["status"] == 0
            assert abs(nll.item() - v_ref) / w.n <= 1e-10, (prec, call)
            np.testing.assert_allclose(grad.cpu().numpy(), g_ref, rtol=1e-8, atol=1e-8 * np.abs(g_ref).max())


def test_noalloc_resets_fallback_state_between_calls():
    """A mixed call on near-duplicate points (rows redone in FP64, their flags
    set in the shared array), then a call with another n and no such rows:
    each must match the workspace entry point, n_fallback included, so the
    flags and counters of one call never leak into the next."""
    torch = cuda_or_skip()
    vst = load_vst()
    rng = np.random.default_rng(12)
    st = si.stations_uniform(120, 12)
    src = rng.choice(120, 80, replace=False)
    dup = st[src] + 1e-5 * rng.standard_normal((80, 2))
    xy1, t1 = si.station_days(np.concatenate([st, dup]), 5)
    o = si.random_order(t1.shape[0], 12)
    xy1, t1 = np.ascontiguousarray(xy1[o]), np.ascontiguousarray(t1[o])
    th1 = oracle.theta_from_ranges(1.0, 0.1, 3.0, 0.5, 1e-5)
    w2 = si.tiny_uniform(m=10)
    th2 = oracle.theta_native(w2.theta)
    m = 10
    cases = []
    for xy, t, th, seed in ((xy1, t1, th1, 1), (w2.xy, w2.t, th2, 2)):
        nn, cnt, _, _ = oracle.knn(xy, t, th, m)
        A, D = oracle.factor(xy, t, th, m, nn, cnt)
        y = oracle.vecchia_sample(m, nn, cnt, A, D, si.standard_normal(t.shape[0], seed))
        cases.append((th, dev(torch, xy, t, y, nn, cnt)))
    nll = torch.empty(1, dtype=torch.float64, device="cuda")
    grad = torch.empty(5, dtype=torch.float64, device="cuda")
    seen = []
    for th, (xy_d, t_d, y_d, nn_d, cnt_d) in cases + cases:
        n = t_d.shape[0]
        ws = vst.Workspace(n, m)
        v_ref, g_ref = vst.vecchia_nll_grad(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=vst.MIXED, ws=ws)
        ref = vst.vst_workspace_status(ws)
        vst.vecchia_nll_grad_noalloc(xy_d, t_d, th, m, nn_d, cnt_d, y_d, precision=vst.MIXED, nll=nll, grad=grad)
        info = vst.vst_noalloc_status()
        assert info["status"] == 0
        assert info["n_fallback"] == ref["n_fallback"]
        assert abs(nll.item() - v_ref.item()) / n <= 1e-10
        np.testing.assert_allclose(grad.cpu().numpy(), g_ref.cpu().numpy(), rtol=1e-8,
                                   atol=1e-8 * np.abs(g_ref.cpu().numpy()).max())
        seen.append(info["n_fallback"])
    assert seen[0] > 0 and seen[1] == 0 and seen[2] == seen[0] and seen[3] == 0


def test_noalloc_rejects_n_beyond_limit():
    torch = cuda_or_skip()
    vst = load_vst()
    th = vst.vst_theta_from_ranges(1.0, 0.1, 3.0, 0.5, 0.05)
    n = vst.NOALLOC_MAX_N + 1
    xy = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    t = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    nn = torch.zeros((n, 1), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(vst.VstError) as e:
        vst.vecchia_nll_grad_noalloc(xy, t, th, 1, nn, cnt, y)
    assert e.value.code == 1 and "VST_NOALLOC_MAX_N" in str(e.value)
