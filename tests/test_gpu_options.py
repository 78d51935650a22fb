"""Per-call options of the _ex entry points and the failure paths.

* The mixed form's FP64 fallback: rows whose condition estimate of the local
  block, (max L_jj / min L_jj)^2, exceeds tau are redone in FP64.  Forced with
  a small tau and with near-duplicate points (default tau and tau = 100); the flagged
  rows must be exactly the rows the oracle's estimate selects (rows within 2%
  of tau, where the FP32 and FP64 estimates may fall on different sides, are
  not compared) and the NLL and gradient must meet the mixed bar, for single
  and batched calls.
* Row ranges: contiguous shards add up to the unsharded NLL and gradient.
* Failure detection without a GPU fault: a bounded wait that runs out gives
  VST_ETIMEOUT and the context stays usable; a singular local block gives
  VST_ENOTSPD with the first bad row.
* The torch.autograd wrapper against central differences and the oracle.

Bars: FP64 |dNLL|/n <= 1e-10; mixed |dNLL|/n <= 1e-6 and, per gradient
component, |dg_j| <= 1e-4 |g_j| + 1e-6 n (the NLL's per-point bar carried to
each n-term sum of the gradient)."""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si
from gpu_util import cuda_or_skip, dev, load_vst

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = cuda_or_skip()
    return torch, load_vst()


def mixed_ok(v, g, vo, go, n):
    assert abs(v - vo) / n <= 1e-6
    assert np.all(np.abs(g - go) <= 1e-4 * np.abs(go) + 1e-6 * n), (g, go)


def expected_flags(est, tau):
    """(rows the oracle's estimate flags, mask of rows safely away from tau)."""
    return est > tau, np.abs(est / tau - 1.0) > 0.02




@pytest.fixture(scope="module")
def tiny(env):
    torch, vst = env
    w = si.tiny_uniform(m=10)
    th = oracle.theta_native(w.theta)
    nn, cnt, _, _ = oracle.knn(w.xy, w.t, th, w.m)
    y = oracle.dense_sample(w.xy, w.t, th, w.z)
    est = oracle.cond_estimates(w.xy, w.t, th, nn, cnt)
    vo, go = oracle.nll_grad(w.xy, w.t, th, w.m, nn, cnt, y)
    xy, t, yd, nnd, cntd = dev(torch, w.xy, w.t, y, nn, cnt)
    return dict(w=w, th=th, nn=nn, cnt=cnt, y=y, est=est, vo=vo, go=go, xy=xy, t=t, yd=yd, nnd=nnd, cntd=cntd)


@pytest.mark.parametrize("tau_kind", ["one", "median"])
def test_forced_fallback_single(env, tiny, tau_kind):
    torch, vst = env
    w, n = tiny["w"], tiny["w"].n
    est = tiny["est"]
    tau = 1.0 if tau_kind == "one" else float(np.median(est[est > 1.0]))
    flags = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
    ws = vst.Workspace(n, w.m)
    v, g = vst.vecchia_nll_grad_ex(tiny["xy"], tiny["t"], tiny["th"], w.m, tiny["nnd"], tiny["cntd"], tiny["yd"],
                                   precision=vst.MIXED, tau=tau, fallback_rows=flags, ws=ws)
    info = vst.vst_workspace_status(ws)
    f = flags.cpu().numpy()
    assert set(np.unique(f).tolist()) <= {0, 1}
    want, safe = expected_flags(est, tau)
    if tau_kind == "one":
        # every row with a neighbour has estimate > 1; FP32 may round the
        # ratio of a nearly uncorrelated block to exactly 1
        safe = safe & (est > 1.0 + 1e-5)
    assert np.array_equal(f[safe].astype(bool), want[safe])
    assert info["n_fallback"] == int(f.sum()) > 0
    mixed_ok(v.item(), g.cpu().numpy(), tiny["vo"], tiny["go"], n)
    if tau_kind == "one":
        # (nearly) every row in FP64: the result is the FP64 form's to rounding
        v64, g64 = vst.vecchia_nll_grad(tiny["xy"], tiny["t"], tiny["th"], w.m, tiny["nnd"], tiny["cntd"],
                                        tiny["yd"], precision=vst.FP64, ws=ws)
        assert f.sum() >= n - 10
        assert abs(v.item() - v64.item()) / n <= 1e-8


def near_duplicates(seed=0, n_st=150, n_days=6, n_dup=40):
    """Stations on [0,1]^2 with n_dup of them repeated at offsets of 1e-5 to
    1e-3 (near-duplicate locations): the local blocks that hold such a pair
    are ill-conditioned when the nugget is small."""
    rng = np.random.default_rng(seed)
    st = si.stations_uniform(n_st, seed)
    src = rng.choice(n_st, n_dup, replace=False)
    ang = rng.random(n_dup) * 2 * np.pi
    rad = 10.0 ** rng.uniform(-5, -3, n_dup)
    dup = st[src] + np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1)
    xy, t = si.station_days(np.concatenate([st, dup]), n_days)
    order = si.random_order(t.shape[0], seed)
    return np.ascontiguousarray(xy[order]), np.ascontiguousarray(t[order])


@pytest.fixture(scope="module")
def dup(env):
    torch, vst = env
    xy, t = near_duplicates()
    th = oracle.theta_from_ranges(1.0, 0.1, 3.0, 0.5, 1e-5)
    m = 10
    nn, cnt, _, _ = oracle.knn(xy, t, th, m)
    A, D = oracle.factor(xy, t, th, m, nn, cnt)
    y = oracle.vecchia_sample(m, nn, cnt, A, D, si.standard_normal(t.shape[0], 3))
    est = oracle.cond_estimates(xy, t, th, nn, cnt)
    vo, go = oracle.nll_grad(xy, t, th, m, nn, cnt, y)
    d = dev(torch, xy, t, y, nn, cnt)
    return dict(xy=xy, t=t, th=th, m=m, nn=nn, cnt=cnt, y=y, est=est, vo=vo, go=go, d=d)


def test_near_duplicates_fall_back(env, dup):
    """Near-duplicate locations with a nugget of 1e-5: about a third of the
    rows have estimates above the default tau = 1e4 and are redone in FP64.
    An unflagged row's FP32 error grows with its estimate (the covariance
    entries are rounded to 2^-24 of sigma1^2 while D_i is ~1e-5 of it), so at
    the default tau the NLL error is a few 1e-6 per point on this data; with
    tau = 100 the 1e-6 bar holds again."""
    torch, vst = env
    xy, t, yd, nnd, cntd = dup["d"]
    n, m = dup["t"].shape[0], dup["m"]
    est = dup["est"]
    assert (est > 1e4).sum() > 20 and (est < 1e4).sum() > n // 2
    ws = vst.Workspace(n, m)
    for tau in (0.0, 100.0):
        flags = torch.zeros(n, dtype=torch.uint8, device="cuda")
        v, g = vst.vecchia_nll_grad_ex(xy, t, dup["th"], m, nnd, cntd, yd, precision=vst.MIXED, tau=tau,
                                       fallback_rows=flags, ws=ws)
        info = vst.vst_workspace_status(ws)
        f = flags.cpu().numpy().astype(bool)
        want, safe = expected_flags(est, tau if tau > 0 else 1e4)
        assert np.array_equal(f[safe], want[safe]), tau
        assert info["n_fallback"] == int(f.sum()) >= int(want[safe].sum())
        if tau == 0.0:
            assert abs(v.item() - dup["vo"]) / n <= 1e-5
            # the plain entry point flags the same rows and returns the same bits
            v2, g2 = vst.vecchia_nll_grad(xy, t, dup["th"], m, nnd, cntd, yd, precision=vst.MIXED, ws=ws)
            assert vst.vst_workspace_status(ws)["n_fallback"] == info["n_fallback"]
            assert v2.item() == v.item() and np.array_equal(g2.cpu().numpy(), g.cpu().numpy())
        else:
            mixed_ok(v.item(), g.cpu().numpy(), dup["vo"], dup["go"], n)


def test_forced_fallback_batched(env, dup):
    """Three datasets: a well-conditioned one, the near-duplicate one, and a
    second well-conditioned one.  Flagged rows must land in their own
    dataset's sums."""
    torch, vst = env
    m = 10
    sets = []
    for seed in (1, 2):
        st = si.stations_uniform(80, seed)
        xy, t = si.station_days(st, 5)
        o = si.random_order(t.shape[0], seed)
        sets.append((np.ascontiguousarray(xy[o]), np.ascontiguousarray(t[o]),
                     oracle.theta_from_ranges(1.0, 0.12 + 0.05 * seed, 2.0 + seed, 0.4, 0.03)))
    sets.insert(1, (dup["xy"], dup["t"], dup["th"]))
    ys, nns, cnts, vals, ests = [], [], [], [], []
    for k, (xy, t, th) in enumerate(sets):
        if k == 1:
            nn, cnt, y = dup["nn"], dup["cnt"], dup["y"]
        else:
            nn, cnt, _, _ = oracle.knn(xy, t, th, m)
            A, D = oracle.factor(xy, t, th, m, nn, cnt)
            y = oracle.vecchia_sample(m, nn, cnt, A, D, si.standard_normal(t.shape[0], 10 + k))
        ys.append(y); nns.append(nn); cnts.append(cnt)
        vals.append(oracle.nll_grad(xy, t, th, m, nn, cnt, y))
        ests.append(oracle.cond_estimates(xy, t, th, nn, cnt))
    ns = [s[1].shape[0] for s in sets]
    offs = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    cat = lambda a: np.ascontiguousarray(np.concatenate(a))
    xy, t, y, nn, cnt, off, thetas = dev(torch, cat([s[0] for s in sets]), cat([s[1] for s in sets]), cat(ys),
                                         cat(nns), cat(cnts), offs, np.stack([s[2] for s in sets]))
    ntot = int(offs[-1])
    ws = vst.BatchedWorkspace(3, ntot, m)
    for tau in (0.0, 100.0, 1.0):
        flags = torch.zeros(ntot, dtype=torch.uint8, device="cuda")
        nll, grad = vst.vecchia_nll_grad_batched_ex(off, thetas, 1.5, xy, t, m, nn, cnt, y, precision=vst.MIXED,
                                                    tau=tau, fallback_rows=flags, ws=ws)
        info = vst.vst_workspace_status(ws)
        f = flags.cpu().numpy().astype(bool)
        nll, grad = nll.cpu().numpy(), grad.cpu().numpy()
        for d in range(3):
            fd = f[offs[d]:offs[d + 1]]
            want, safe = expected_flags(ests[d], 1e4 if tau == 0.0 else tau)
            if tau == 1.0:
                safe = safe & (ests[d] > 1.0 + 1e-5)
            assert np.array_equal(fd[safe], want[safe]), (tau, d)
            if tau > 0 or d != 1:  # the default tau is too loose for the 1e-6 bar on set 1 (see above)
                mixed_ok(nll[d], grad[d], vals[d][0], vals[d][1], ns[d])
        assert info["n_fallback"] == int(f.sum())
        if tau == 0.0:
            assert f[offs[1]:offs[2]].sum() > 20 and f[:offs[1]].sum() == 0 and f[offs[2]:].sum() == 0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_row_range_shards_add_up(env, tiny, prec):
    torch, vst = env
    w, n = tiny["w"], tiny["w"].n
    p = vst.FP64 if prec == "fp64" else vst.MIXED
    args = (tiny["xy"], tiny["t"], tiny["th"], w.m, tiny["nnd"], tiny["cntd"], tiny["yd"])
    ws = vst.Workspace(n, w.m)
    v, g = vst.vecchia_nll_grad(*args, precision=p, ws=ws)
    v, g = v.item(), g.cpu().numpy()
    for cuts in ([0, 777, n], [0, 1, 2, 1000, 1999, n]):
        sv, sg = 0.0, np.zeros(5)
        for b, e in zip(cuts[:-1], cuts[1:]):
            vb, gb = vst.vecchia_nll_grad_ex(*args, precision=p, row_begin=b, row_end=e, ws=ws)
            vst.vst_workspace_status(ws)
            sv += vb.item()
            sg += gb.cpu().numpy()
        assert abs(sv - v) <= 1e-13 * abs(v)
        assert np.all(np.abs(sg - g) <= 1e-13 * np.abs(g) + 1e-13 * np.abs(g).max())
    # a shard's terms are the oracle's terms of its rows
    vb, gb = vst.vecchia_nll_grad_ex(*args, precision=vst.FP64, row_begin=500, row_end=1500, ws=ws)
    rows = np.arange(500, 1500)
    _, _, terms = oracle.nll_grad(w.xy, w.t, tiny["th"], w.m, tiny["nn"], tiny["cnt"], tiny["y"], terms=True)
    ref = 0.5 * 1000 * np.log(2 * np.pi) + oracle.nll(w.xy, w.t, tiny["th"], w.m, tiny["nn"], tiny["cnt"],
                                                      tiny["y"], terms=True)[1][rows].sum()
    assert abs(vb.item() - ref) / 1000 <= 1e-10
    np.testing.assert_allclose(gb.cpu().numpy(), terms[rows].sum(0), rtol=1e-8, atol=1e-9 * np.abs(terms).sum())
    # an empty range and a bad range
    ve, ge = vst.vecchia_nll_grad_ex(*args, precision=p, row_begin=300, row_end=300, ws=ws)
    assert ve.item() == 0.0 and not ge.cpu().numpy().any()
    with pytest.raises(vst.VstError):
        vst.vecchia_nll_grad_ex(*args, precision=p, row_begin=10, row_end=n + 1, ws=ws)


def test_bounded_wait_runs_out(env):
    """Vecchia sampling waits (bounded) on predecessor rows other warps are
    computing.  With a limit of one poll most such waits run out: the call
    records VST_ETIMEOUT in the workspace, and the next call on the same
    context works."""
    torch, vst = env
    w = si.box_uniform(m=20, n_days=20)
    th = oracle.theta_native(w.theta)
    xy, t, z = dev(torch, w.xy, w.t, w.z)
    ws = vst.Workspace(w.n, w.m)
    nn, cnt = vst.vif_build_neighbors(xy, t, th, w.m, ws=ws)
    vst.vst_workspace_status(ws)
    vst.vecchia_sample_ex(xy, t, th, w.m, nn, cnt, z, wait_limit=1, ws=ws)
    info = vst.vst_workspace_status(ws, raise_on_error=False)
    assert info["status"] == 4  # VST_ETIMEOUT
    assert 0 < info["bad_row"] < w.n
    y = vst.vecchia_sample(xy, t, th, w.m, nn, cnt, z, ws=ws)
    assert vst.vst_workspace_status(ws)["status"] == 0
    assert torch.isfinite(y).all()
    # the sample is the whitening inverse of the FP64 factor: the NLL's
    # residual part is exactly 1/2 sum z^2
    A, D = vst.vecchia_factor(xy, t, th, w.m, nn, cnt, precision=vst.FP64, ws=ws)
    v = vst.vecchia_nll(xy, t, th, w.m, nn, cnt, y, precision=vst.FP64, ws=ws).item()
    ref = 0.5 * w.n * np.log(2 * np.pi) + 0.5 * torch.log(D).sum().item() + 0.5 * float((w.z ** 2).sum())
    assert abs(v - ref) / w.n <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_singular_block_reports_not_spd(env, prec):
    """A point repeated exactly (same location and day) with no nugget: the
    block of the repeat and its only neighbour, the original, is [[s, s],
    [s, s]], whose second pivot is exactly 0.  The call reports VST_ENOTSPD
    at the first such row (the mixed form flags the row and its FP64 redo
    fails the same way)."""
    torch, vst = env
    rng = np.random.default_rng(8)
    n = 300
    xy = rng.random((n, 2))
    t = rng.integers(0, 5, n).astype(np.float64)
    for r in (137, 211):
        xy[r], t[r] = xy[r - 1], t[r - 1]
    nn = np.full((n, 1), -1, dtype=np.int32)
    nn[1:, 0] = np.arange(n - 1)
    cnt = np.minimum(np.arange(n), 1).astype(np.int32)
    th = oracle.theta_from_ranges(1.0, 0.1, 3.0, 0.5, 0.0)
    xyd, td, yd, nnd, cntd = dev(torch, xy, t, rng.standard_normal(n), nn, cnt)
    ws = vst.Workspace(n, 1)
    vst.vecchia_nll_grad(xyd, td, th, 1, nnd, cntd, yd, precision=vst.FP64 if prec == "fp64" else vst.MIXED,
                         ws=ws)
    info = vst.vst_workspace_status(ws, raise_on_error=False)
    assert info["status"] == 3  # VST_ENOTSPD
    assert info["bad_row"] == 137
    # the context stays usable: without the repeats the call succeeds
    nn2, cnt2 = dev(torch, nn, cnt)
    xy2 = xy.copy()
    xy2[137] += 0.01
    xy2[211] += 0.01
    vst.vecchia_nll_grad(dev(torch, xy2)[0], td, th, 1, nn2, cnt2, yd, precision=vst.FP64, ws=ws)
    assert vst.vst_workspace_status(ws)["status"] == 0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_autograd_wrapper(env, tiny, prec):
    """VecchiaNLL.apply(...).backward() gives the gradient of the NLL with
    respect to (sigma1sq, c, a, gamma, nugget): central differences of the
    NLL (h = 1e-6 relative, FP64) and the oracle's gradient."""
    torch, vst = env
    w, n = tiny["w"], tiny["w"].n
    th = np.asarray(tiny["th"])
    p = vst.FP64 if prec == "fp64" else vst.MIXED
    theta5 = torch.tensor(th[:5], dtype=torch.float64, requires_grad=True)
    ws = vst.Workspace(n, w.m)
    out = vst.VecchiaNLL.apply(theta5, tuple(th[5:]), tiny["xy"], tiny["t"], tiny["yd"], tiny["nnd"],
                               tiny["cntd"], w.m, p, ws)
    (3.0 * out).backward()
    g = theta5.grad.numpy() / 3.0
    assert out.item() == pytest.approx(tiny["vo"], abs=(1e-10 if prec == "fp64" else 1e-6) * n)
    if prec == "fp64":
        np.testing.assert_allclose(g, tiny["go"], rtol=1e-8, atol=1e-8 * np.abs(tiny["go"]).max())
        for q in range(5):
            e = 1e-6 * abs(th[q])
            tp, tm = th.copy(), th.copy()
            tp[q] += e
            tm[q] -= e
            fp = vst.vecchia_nll(tiny["xy"], tiny["t"], tp, w.m, tiny["nnd"], tiny["cntd"], tiny["yd"], ws=ws).item()
            fm = vst.vecchia_nll(tiny["xy"], tiny["t"], tm, w.m, tiny["nnd"], tiny["cntd"], tiny["yd"], ws=ws).item()
            assert g[q] == pytest.approx((fp - fm) / (2 * e), rel=1e-5, abs=1e-4)
    else:
        mixed_ok(out.item(), g, tiny["vo"], tiny["go"], n)
