"""C-ABI library: it builds, loads, exports every symbol include/vst.h declares,
and its host-only entry points validate arguments.  No compute call (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def vst():
    from paper_2602_03609_gb300 import build
    build.build()
    import paper_2602_03609_gb300 as p
    return p


def test_exports_every_declared_symbol(vst):
    names = declared_functions()
    assert {"vif_build_neighbors", "vecchia_factor", "vecchia_nll", "vecchia_nll_grad"} <= set(names)
    L = ctypes.CDLL(vst.LIB_PATH)
    for nm in names:
        assert hasattr(L, nm), nm


def test_noalloc_scratch_size_matches_its_layout(vst):
    # header 256 B, FP64 and FP32 lag tables (1024 lags x 32 B and x 16 B),
    # two per-warp partial buffers (65,536 warps x 8 doubles), one flag byte
    # and one 32-byte mixed-form record per point (2^21 points)
    n = vst.NOALLOC_MAX_N
    assert n == 1 << 21
    expect = 256 + 1024 * 32 + 1024 * 16 + 2 * 65536 * 8 * 8 + n + 32 * n
    assert vst.vst_noalloc_scratch_bytes() == expect == 77_644_032


def test_theta_from_ranges_matches_oracle(vst):
    for args in [(1, 0.1, 3, 0.5, 0.05, 0.4, 0.2, 1.5), (2, 0.08, 5, 0.9, 0.1, 0.7, 0.1, 0.5),
                 (1, 0.3, 1, 0.1, 0.2, 0.4, 0.2, 2.5)]:
        np.testing.assert_allclose(vst.vst_theta_from_ranges(*args), oracle.theta_from_ranges(*args), rtol=1e-13)
    with pytest.raises(vst.VstError):
        vst.vst_theta_from_ranges(1, -0.1, 3, 0.5, 0.05)
    with pytest.raises(vst.VstError):
        vst.vst_theta_from_ranges(1, 0.1, 3, 0.5, 0.05, nu=1.0)


def test_workspace_size_monotone(vst):
    a = vst.vst_workspace_size(1000, 10)
    b = vst.vst_workspace_size(100000, 10)
    c = vst.vst_workspace_size(100000, 30)
    assert 0 < a < b < c
    assert vst.vst_workspace_size(0, 0) > 0


def test_vif_grad_workspace_holds_the_tensor_core_scratch(vst):
    # the mixed VIF gradient's J = H^T U: both operands transposed into three
    # BF16 parts [3][kp][np] (kp = k rounded up to 256, np = n rounded up to
    # 64) and up to 16 FP64 k x k segment partials, beyond the NLL's workspace
    for n, m, k in ((1000, 10, 24), (30000, 30, 1000), (1108140, 30, 1000), (5, 4, 257)):
        kp = (k + 255) // 256 * 256
        np_ = (n + 63) // 64 * 64
        extra = vst.vst_workspace_size_vif_grad(n, m, k) - vst.vst_workspace_size(n, m, k)
        assert extra >= 2 * 3 * kp * np_ * 2 + 16 * k * k * 8, (n, m, k)


def test_host_validation_without_gpu(vst):
    L = vst.lib()
    th = vst._Theta(*vst.vst_theta_from_ranges(1, 0.1, 3, 0.5, 0.05))
    pts = vst._Points(None, None, 10)
    # m beyond the supported maximum
    rc = L.vecchia_nll(ctypes.byref(pts), ctypes.byref(th), 40, None, None, None, None, 0, None, None, 0, None)
    assert rc == 1 and b"m=40" in L.vst_last_error()
    # invalid covariance parameters
    bad = vst._Theta(1.0, -1.0, 1.0, 0.5, 0.05, 0.4, 0.2, 1.5)
    rc = L.vecchia_nll(ctypes.byref(pts), ctypes.byref(bad), 10, None, None, None, None, 0, None, None, 0, None)
    assert rc == 1
    # unsupported smoothness
    bad = vst._Theta(1.0, 1.0, 1.0, 0.5, 0.05, 0.4, 0.2, 1.0)
    rc = L.vecchia_nll(ctypes.byref(pts), ctypes.byref(bad), 10, None, None, None, None, 0, None, None, 0, None)
    assert rc == 1 and b"nu" in L.vst_last_error()
    # NULL arrays
    rc = L.vecchia_nll_grad(ctypes.byref(pts), ctypes.byref(th), 10, None, None, None, None, 0, None, None,
                            None, 0, None)
    assert rc == 1
    # workspace too small (non-NULL, aligned dummy address; never dereferenced)
    pts = vst._Points(256, 512, 10)
    rc = L.vecchia_factor(ctypes.byref(pts), ctypes.byref(th), 5, None, 1024, 2048, 0, 4096, 8192, 256, 16,
                          None)
    assert rc == 2
    # the VIF gradient: a bad precision, and its own (larger) workspace;
    # too many inducing points
    ind = vst._Inducing(256, 512, 5)
    rc = L.vecchia_nll_grad(ctypes.byref(pts), ctypes.byref(th), 5, ctypes.byref(ind), 1024, 2048, 4096, 9, 8192,
                            8448, 256, 1 << 40, None)
    assert rc == 1 and b"precision" in L.vst_last_error()
    need = L.vst_workspace_size_vif_grad(10, 5, 5)
    assert need > L.vst_workspace_size(10, 5, 5)
    rc = L.vecchia_nll_grad(ctypes.byref(pts), ctypes.byref(th), 5, ctypes.byref(ind), 1024, 2048, 4096, 0, 8192,
                            8448, 256, need - 1, None)
    assert rc == 2
    big = vst._Inducing(256, 512, 1 << 20)
    rc = L.vif_build_neighbors(ctypes.byref(pts), ctypes.byref(th), 5, ctypes.byref(big), 1024, 2048, None, 0,
                               256, 1 << 40, None)
    assert rc == 1 and b"inducing" in L.vst_last_error()


def test_gram_tc_workspace_size_and_argument_checks(vst):
    # header 256 B; two operands, each its transposed parts (3 parts x kp x
    # np BF16, kp = kc rounded up to 256, np = n rounded up to 128), an int16
    # exponent per column and 128-row block and an int32 one per column; then
    # 16 segments of kc x kc doubles
    n, kc = 1000, 300
    kp, np_ = 512, 1024
    opb = 2 * 3 * kp * np_ + 2 * (np_ // 128) * kp + 4 * kp
    expect = 256 + 2 * opb + 8 * 16 * kc * kc
    assert vst.vst_workspace_size_gram_tc(n, kc) == expect
    assert vst.vst_workspace_size_gram_tc(n, 0) == 0
    L = vst.lib()
    fake = ctypes.c_void_p(256)
    for nn_, kc_ in [(n, 0), (-1, kc), (n, 20000)]:
        rc = L.vif_gram_tc(nn_, kc_, fake, max(kc_, 1), None, 0, fake, fake, 1 << 40, None)
        assert rc == 1, (nn_, kc_)  # VST_EINVAL, before any device work
    rc = L.vif_gram_tc(n, kc, fake, kc - 1, None, 0, fake, fake, 1 << 40, None)
    assert rc == 1
    rc = L.vif_gram_tc(n, kc, fake, kc, None, 0, fake, fake, expect - 1, None)
    assert rc == 2  # VST_ENOMEM
