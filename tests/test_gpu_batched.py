"""Batched driver: independent datasets with their own parameters and sizes in
one persistent launch, its CUDA graph, the launch-shape autotuner, and the
central-difference gradient check of the batched workload (h = 1e-6, FP64)."""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si
from gpu_util import cuda_or_skip, dev, load_vst

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    torch = cuda_or_skip()
    vst = load_vst()
    sets = si.batched(seed=7, n_sets=6, m=10, n_days=10, n_lo=300, n_hi=1500)
    m = 10
    ths, nns, cnts, ys, vals = [], [], [], [], []
    for w in sets:
        th = oracle.theta_native(w.theta)
        nn, cnt, _, _ = oracle.knn(w.xy, w.t, th, m)
        A, D = oracle.factor(w.xy, w.t, th, m, nn, cnt)
        y = oracle.vecchia_sample(m, nn, cnt, A, D, w.z)
        ths.append(th); nns.append(nn); cnts.append(cnt); ys.append(y)
        vals.append(oracle.nll_grad(w.xy, w.t, th, m, nn, cnt, y))
    offs = np.concatenate([[0], np.cumsum([w.n for w in sets])]).astype(np.int64)
    cat = lambda arrs: np.ascontiguousarray(np.concatenate(arrs))
    xy, t, y, nn, cnt, off, thetas = dev(torch, cat([w.xy for w in sets]), cat([w.t for w in sets]), cat(ys),
                                         cat(nns), cat(cnts), offs, np.stack(ths))
    return dict(torch=torch, vst=vst, sets=sets, m=m, ths=ths, vals=vals, offs=offs, xy=xy, t=t, y=y, nn=nn,
                cnt=cnt, off=off, thetas=thetas, nns=nns, cnts=cnts, ys=ys)


def check_against_oracle(b, nll, grad, tol):
    for d, w in enumerate(b["sets"]):
        vo, go = b["vals"][d]
        assert abs(nll[d] - vo) / w.n <= tol, d
        assert np.all(np.abs(grad[d] - go) <= max(tol * 1e2, 1e-8) * np.maximum(np.abs(go), 1.0) * w.n ** 0.5), d


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-6)])
def test_batched_matches_oracle_and_single_calls(batch, prec, tol):
    vst, b = batch["vst"], batch
    ws = vst.BatchedWorkspace(len(b["sets"]), b["t"].shape[0], b["m"])
    nll, grad = vst.vecchia_nll_grad_batched(b["off"], b["thetas"], 1.5, b["xy"], b["t"], b["m"], b["nn"], b["cnt"],
                                             b["y"], precision=prec, ws=ws)
    vst.vst_workspace_status(ws)
    nll, grad = nll.cpu().numpy(), grad.cpu().numpy()
    check_against_oracle(b, nll, grad, tol)
    # the same datasets one by one through the single-dataset entry point
    torch = b["torch"]
    for d, w in enumerate(b["sets"]):
        xy, t, y, nn, cnt = dev(torch, w.xy, w.t, b["ys"][d], b["nns"][d], b["cnts"][d])
        v, g = vst.vecchia_nll_grad(xy, t, b["ths"][d], b["m"], nn, cnt, y, precision=prec)
        assert abs(v.item() - nll[d]) / w.n <= 1e-12
        np.testing.assert_allclose(g.cpu().numpy(), grad[d], rtol=1e-9, atol=1e-9)


def test_graph_replay_and_parameter_update(batch):
    vst, b, torch = batch["vst"], batch, batch["torch"]
    ns = len(b["sets"])
    ws = vst.BatchedWorkspace(ns, b["t"].shape[0], b["m"])
    thetas = b["thetas"].clone()
    nll = torch.empty(ns, dtype=torch.float64, device="cuda")
    grad = torch.empty((ns, 5), dtype=torch.float64, device="cuda")
    gr = vst.BatchedGraph(b["off"], thetas, 1.5, b["xy"], b["t"], b["m"], b["nn"], b["cnt"], b["y"], vst.FP64, nll,
                          grad, ws)
    ref = nll.clone(), grad.clone()
    for _ in range(2):
        nll.zero_(); grad.zero_()
        gr.launch()
        torch.cuda.synchronize()
        assert torch.equal(nll, ref[0]) and torch.equal(grad, ref[1])
    # update the parameters in place and replay: equals a direct evaluation
    thetas[:, 4] *= 1.3
    thetas[:, 1] *= 0.9
    gr.launch()
    torch.cuda.synchronize()
    n2, g2 = vst.vecchia_nll_grad_batched(b["off"], thetas, 1.5, b["xy"], b["t"], b["m"], b["nn"], b["cnt"], b["y"],
                                          precision=vst.FP64)
    assert torch.equal(nll, n2) and torch.equal(grad, g2)
    assert not torch.equal(nll, ref[0])
    gr.close()


def test_central_differences_batched_fp64(batch):
    vst, b, torch = batch["vst"], batch, batch["torch"]
    ns = len(b["sets"])
    ws = vst.BatchedWorkspace(ns, b["t"].shape[0], b["m"])
    thetas = b["thetas"].clone()
    nll = torch.empty(ns, dtype=torch.float64, device="cuda")
    grad = torch.empty((ns, 5), dtype=torch.float64, device="cuda")
    gr = vst.BatchedGraph(b["off"], thetas, 1.5, b["xy"], b["t"], b["m"], b["nn"], b["cnt"], b["y"], vst.FP64, nll,
                          grad, ws)
    gr.launch()
    g0 = grad.cpu().numpy().copy()
    base = thetas.clone()
    for p in range(5):
        h = 1e-6 * torch.clamp(base[:, p].abs(), min=1.0)
        thetas.copy_(base); thetas[:, p] += h
        gr.launch(); fp = nll.cpu().numpy().copy()
        thetas.copy_(base); thetas[:, p] -= h
        gr.launch(); fm = nll.cpu().numpy().copy()
        fd = (fp - fm) / (2 * h.cpu().numpy())
        np.testing.assert_allclose(g0[:, p], fd, rtol=2e-5, atol=2e-4)
    gr.close()


def test_autotuner_keeps_results(batch):
    vst, b, torch = batch["vst"], batch, batch["torch"]
    vst.vst_autotune_clear()
    n0, g0 = vst.vecchia_nll_grad_batched(b["off"], b["thetas"], 1.5, b["xy"], b["t"], b["m"], b["nn"], b["cnt"],
                                          b["y"], precision=vst.MIXED)
    bps, chunk, ms = vst.vst_autotune_nll_grad_batched(b["off"], b["thetas"], 1.5, b["xy"], b["t"], b["m"], b["nn"],
                                                       b["cnt"], b["y"], precision=vst.MIXED)
    assert bps in (0, 1, 2, 3) and chunk in (1, 4, 16, 64) and ms > 0
    n1, g1 = vst.vecchia_nll_grad_batched(b["off"], b["thetas"], 1.5, b["xy"], b["t"], b["m"], b["nn"], b["cnt"],
                                          b["y"], precision=vst.MIXED)
    np.testing.assert_allclose(n1.cpu().numpy(), n0.cpu().numpy(), rtol=1e-12)
    np.testing.assert_allclose(g1.cpu().numpy(), g0.cpu().numpy(), rtol=1e-6, atol=1e-6)
    # single-dataset tuner
    w = b["sets"][0]
    xy, t, y, nn, cnt = dev(torch, w.xy, w.t, b["ys"][0], b["nns"][0], b["cnts"][0])
    r = vst.vst_autotune_nll_grad(xy, t, b["ths"][0], b["m"], nn, cnt, y, precision=vst.MIXED)
    v, _ = vst.vecchia_nll_grad(xy, t, b["ths"][0], b["m"], nn, cnt, y, precision=vst.MIXED)
    assert abs(v.item() - b["vals"][0][0]) / w.n <= 1e-6
    vst.vst_autotune_clear()


def test_invalid_dataset_parameters_reported(batch):
    vst, b = batch["vst"], batch
    ns = len(b["sets"])
    thetas = b["thetas"].clone()
    thetas[3, 1] = -1.0  # negative spatial decay in dataset 3
    ws = vst.BatchedWorkspace(ns, b["t"].shape[0], b["m"])
    vst.vecchia_nll_grad_batched(b["off"], thetas, 1.5, b["xy"], b["t"], b["m"], b["nn"], b["cnt"], b["y"], ws=ws)
    with pytest.raises(vst.VstError) as e:
        vst.vst_workspace_status(ws)
    assert e.value.code == 1 and e.value.info["bad_row"] == 3
