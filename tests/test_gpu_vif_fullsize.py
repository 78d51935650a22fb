"""The VIF model at the bench workload's full size (continental: 1,108,140
points, k = 1000 inducing points from seeded space-time kMeans++ with Lloyd
steps on a 50,000-point subsample, m = 30), in the configuration bench.py
times: the residual-correlation neighbour search (Sect. 4.3 with the
selection of Sect. 4.4.1) checked against the oracle's brute force on
sampled rows (bit-exact sets except cut-off ties, 1e-12 relative), and the
mixed-precision VIF NLL against the FP64 one (|dNLL|/n <= 1e-6)."""
import numpy as np
import pytest

import oracle
import oracle.vif as ovif
import synthetic_inputs as si
from gpu_util import check_neighbours, cuda_or_skip, dev, load_vst

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vfull():
    torch = cuda_or_skip()
    vst = load_vst()
    w = si.continental()
    th = oracle.theta_native(w.theta)
    r = np.random.default_rng(5).choice(w.n, 50000, replace=False)
    r.sort()
    sub = type(w)(name="sub", xy=w.xy[r], t=w.t[r], z=w.z[r], theta=w.theta, m=w.m, order=None)
    xyk, tk = si.inducing_points(sub, 1000, seed=11, lloyd_iters=10)
    xy, t, z, xykd, tkd = dev(torch, w.xy, w.t, w.z, xyk, tk)
    ws = vst.Workspace(w.n, w.m, 1000)
    nn, cnt = vst.vif_build_neighbors(xy, t, th, w.m, ws=ws, inducing=(xykd, tkd))
    info = vst.vst_workspace_status(ws)
    return dict(torch=torch, vst=vst, w=w, th=th, xyk=xyk, tk=tk, xy=xy, t=t, z=z, ind=(xykd, tkd), ws=ws, nn=nn,
                cnt=cnt, info=info)


def test_residual_neighbours_sampled_rows(vfull):
    w, th = vfull["w"], vfull["th"]
    U, r = ovif.lowrank_rows(w.xy, w.t, vfull["xyk"], vfull["tk"], th)
    rng = np.random.default_rng(1)
    rows = np.unique(np.concatenate([np.arange(0, 40, 7), rng.choice(w.n, 20, replace=False), [w.n - 1]]))
    nn_o, cnt_o, rm, rm1 = ovif.knn_rows(w.xy, w.t, th, U, r, w.m, rows)
    nn_g = vfull["nn"].cpu().numpy()[rows]
    cnt_g = vfull["cnt"].cpu().numpy()[rows]
    check_neighbours(nn_g, cnt_g, nn_o, cnt_o, rm, rm1)


def test_vif_nll_full_size_mixed_vs_fp64(vfull):
    vst = vfull["vst"]
    w, th = vfull["w"], vfull["th"]
    ws = vfull["ws"]
    args = (vfull["xy"], vfull["t"], th, w.m, vfull["nn"], vfull["cnt"], vfull["z"])
    v64 = vst.vecchia_nll(*args, precision=vst.FP64, ws=ws, inducing=vfull["ind"]).item()
    vst.vst_workspace_status(ws)
    vmx = vst.vecchia_nll(*args, precision=vst.MIXED, ws=ws, inducing=vfull["ind"]).item()
    vst.vst_workspace_status(ws)
    assert np.isfinite(v64)
    assert abs(vmx - v64) / w.n <= 1e-6
