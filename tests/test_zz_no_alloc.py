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
