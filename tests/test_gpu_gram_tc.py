"""The tensor-core contraction over the points (vif_gram_tc: the W^T W, W^T e
and e^T e of the VIF's Woodbury form, Sect. 4.3, and the gradient's k x k
contractions) against the plain FP64 product A^T B of the same FP32 values.

In each block of 128 rows, column c gets the exponent E with
max |A[i][c]| < 2^E over the block; values are cut into three 9-bit
fixed-point BF16 parts of 2^(E - 8).  Pins:
(1) values that the parts hold exactly (integer multiples of 2^(E - 8)) give
    the product bit for bit: the leading part products are integers below
    2^16 and their sums over each 128-row block integers below 2^23, exact
    whatever the tensor core's rounding;
(2) general values meet the split's bound per element: every dropped product
    and remainder is at most 2^-9 units of 2^(E_a + E_b - 16) per row (E the
    block's exponents, at most the column's largest, Eg), and the correction
    sums' FP32 rounding stays below 2^-12 units per row, so
    |dC_ab| <= n 2^(Eg_a + Eg_b - 16) 2^-8; on rows of very different scales
    the typical error stays within a small factor of an FP32 GEMM's;
(3) a sum of squares over 200,000 rows (the e^T e of the Woodbury form)
    carries no systematic error: relative error <= 1e-9, where a floating
    split whose leading accumulator is not round-to-nearest is biased by
    ~1e-7."""
import numpy as np
import pytest

from gpu_util import cuda_or_skip, load_vst

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = cuda_or_skip()
    return torch, load_vst()


def col_exp(A):
    """E_c with max |A[:, c]| < 2^E_c (FP32 exponent of the column maximum)."""
    mx = np.abs(A).max(axis=0).astype(np.float32)
    bits = mx.view(np.uint32)
    return ((bits >> 23) & 0xFF).astype(np.int64) - 126


def fixed_point_matrix(rng, n, kc):
    e = rng.integers(-6, 7, kc)
    q = rng.integers(-255, 256, (n, kc))
    q[rng.integers(0, n), :] = 255  # column maximum in [2^(E-1), 2^E): exponent E_c = e_c
    A = (q * np.ldexp(1.0, e - 8)[None, :]).astype(np.float32)
    assert np.array_equal(col_exp(A), e)
    return A


def test_exact_on_fixed_point_values(env):
    torch, vst = env
    rng = np.random.default_rng(3)
    n, kc = 20011, 300  # ragged in the 128-row blocks, the 64-row tiles and the 128-column tiles
    A = fixed_point_matrix(rng, n, kc)
    B = fixed_point_matrix(rng, n, kc)
    ref_ab = A.astype(np.float64).T @ B.astype(np.float64)  # integers times powers of two, exact
    ref_aa = A.astype(np.float64).T @ A.astype(np.float64)
    # A with strided rows (row stride kc + 5 floats)
    Ad = torch.zeros((n, kc + 5), dtype=torch.float32, device="cuda")
    Ad[:, :kc] = torch.from_numpy(A).cuda()
    Bd = torch.from_numpy(B).cuda()
    ws = vst._RawWorkspace(vst.vst_workspace_size_gram_tc(n, kc))
    C = vst.vif_gram_tc(Ad[:, :kc], Bd, ws=ws)
    vst.vst_workspace_status(ws)
    assert np.array_equal(C.cpu().numpy(), ref_ab)
    S = vst.vif_gram_tc(Ad[:, :kc], None, ws=ws)
    vst.vst_workspace_status(ws)
    assert np.array_equal(S.cpu().numpy(), ref_aa)


def test_error_bound_general_values(env):
    torch, vst = env
    rng = np.random.default_rng(4)
    n, kc = 30000, 257  # kp = 512: 2 x 2 tiles, the last one almost empty
    # rows of very different scales (as W = D^{-1/2} B U), columns of different scales
    A = (rng.standard_normal((n, kc)) * np.exp(rng.normal(0, 1.5, n))[:, None]
         * np.exp(rng.normal(0, 2, kc))[None, :]).astype(np.float32)
    B = (rng.standard_normal((n, kc)) * np.exp(rng.normal(0, 1.5, n))[:, None]).astype(np.float32)
    A[:, 7] = 0.0  # an all-zero column
    ea, eb = col_exp(A), col_exp(B)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    for Bx, Bn, e2 in ((Bd, B, ea[:, None] + eb[None, :]), (None, A, ea[:, None] + ea[None, :])):
        C = vst.vif_gram_tc(Ad, Bx).cpu().numpy()
        ref = A.astype(np.float64).T @ Bn.astype(np.float64)
        assert np.all(np.abs(C - ref) <= n * 2.0 ** -8 * np.ldexp(1.0, e2 - 16))
        if Bx is None:
            assert np.array_equal(C, C.T)
        assert np.all(C[7] == 0.0)
        # typical error against an FP32 GEMM of the same values
        c32 = (A.T @ Bn).astype(np.float64)
        big = np.abs(ref) > 1e-3 * np.abs(ref).max()
        rel = np.abs(C - ref)[big] / np.abs(ref)[big]
        rel32 = np.abs(c32 - ref)[big] / np.abs(ref)[big]
        assert np.median(rel) <= 10 * np.median(rel32), (np.median(rel), np.median(rel32))


def test_sum_of_squares_unbiased(env):
    torch, vst = env
    rng = np.random.default_rng(5)
    n, kc = 200000, 8
    A = rng.standard_normal((n, kc)).astype(np.float32)
    ref = (A.astype(np.float64) ** 2).sum(0)
    C = vst.vif_gram_tc(torch.from_numpy(A).cuda(), None).cpu().numpy()
    rel = (np.diag(C) - ref) / ref
    assert np.all(np.abs(rel) <= 1e-9), rel


def test_empty_and_tiny(env):
    torch, vst = env
    A = torch.zeros((0, 5), dtype=torch.float32, device="cuda")
    C = vst.vif_gram_tc(A, None)
    assert torch.count_nonzero(C).item() == 0
    A1 = torch.tensor([[1.5, -2.0, 0.25]], dtype=torch.float32, device="cuda")
    C1 = vst.vif_gram_tc(A1, None).cpu().numpy()
    a = np.array([1.5, -2.0, 0.25])
    assert np.array_equal(C1, np.outer(a, a))
