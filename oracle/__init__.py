"""CPU oracle for the Vecchia / VIF space-time likelihood (arXiv 2602.03609).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_2602_03609_gb300``) and never imports it.

The arithmetic lives in ``vecchia_oracle.cpp`` (plain FP64 C++, every
function citing the passage of the paper it writes out); this module only
marshals numpy arrays through ctypes.  ``vif.py`` holds the VIF oracle in
numpy.  Parity status per function is listed in the C++ source.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_matern.restype = ctypes.c_double
        L.orc_matern.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_cov.restype = ctypes.c_double
        L.orc_cov.argtypes = [_D, ctypes.c_double, ctypes.c_double]
        L.orc_cov_grad.restype = None
        L.orc_cov_grad.argtypes = [_D, ctypes.c_double, ctypes.c_double, _D]
        L.orc_theta_from_ranges.restype = ctypes.c_int
        L.orc_theta_from_ranges.argtypes = [ctypes.c_double] * 8 + [_D]
        L.orc_knn_rows.restype = None
        L.orc_knn_rows.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_int, ctypes.c_int64, _I64,
                                   _I32, _I32, _D, _D, ctypes.c_int]
        L.orc_factor.restype = ctypes.c_int64
        L.orc_factor.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_int, _I32, _I32, _D, _D, ctypes.c_int]
        L.orc_factor_rows.restype = None
        L.orc_factor_rows.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_int, ctypes.c_int64, _I64, _I32, _I32,
                                      _D, _D, ctypes.c_int]
        L.orc_nll_grad_rows.restype = ctypes.c_double
        L.orc_nll_grad_rows.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_int, ctypes.c_int64, _I64, _I32, _I32,
                                        _D, _D, ctypes.c_int]
        L.orc_cover_tree_build.restype = ctypes.c_void_p
        L.orc_cover_tree_build.argtypes = [ctypes.c_int64, _D, _D, _D]
        L.orc_cover_tree_free.restype = None
        L.orc_cover_tree_free.argtypes = [ctypes.c_void_p]
        L.orc_cover_tree_depth.restype = ctypes.c_int
        L.orc_cover_tree_depth.argtypes = [ctypes.c_void_p]
        L.orc_cover_tree_structure.restype = None
        L.orc_cover_tree_structure.argtypes = [ctypes.c_void_p, ctypes.c_int64, _I32, _I64]
        L.orc_knn_cover_tree.restype = None
        L.orc_knn_cover_tree.argtypes = [ctypes.c_void_p, ctypes.c_int64, _D, _D, _D, ctypes.c_int, ctypes.c_int64,
                                         _I64, _I32, _I32, _D, _D, ctypes.c_int]
        L.orc_nll.restype = ctypes.c_double
        L.orc_nll.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_int, _I32, _I32, _D, _D, ctypes.c_int]
        L.orc_nll_grad.restype = ctypes.c_double
        L.orc_nll_grad.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_int, _I32, _I32, _D, _D, _D,
                                   ctypes.c_int]
        L.orc_vecchia_sample.restype = None
        L.orc_vecchia_sample.argtypes = [ctypes.c_int64, ctypes.c_int, _I32, _I32, _D, _D, _D, _D]
        L.orc_dense_nll.restype = ctypes.c_double
        L.orc_dense_nll.argtypes = [ctypes.c_int64, _D, _D, _D, _D, _D]
        L.orc_dense_sample.restype = ctypes.c_int
        L.orc_dense_sample.argtypes = [ctypes.c_int64, _D, _D, _D, _D, _D]
        L.orc_cov_matrix.restype = None
        L.orc_cov_matrix.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_int64, _D, _D, _D, _D]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def theta_from_ranges(sigma2, range_s, range_t, gamma, nugget, alpha=0.4, delta=0.2, nu=1.5) -> np.ndarray:
    """Native parameters (sigma1^2, c, a, gamma, nugget, alpha, delta, nu)."""
    out = np.zeros(8)
    rc = lib().orc_theta_from_ranges(sigma2, range_s, range_t, gamma, nugget, alpha, delta, nu, _d(out))
    if rc != 0:
        raise ValueError("invalid ranges")
    return out


def theta_native(rt) -> np.ndarray:
    """From a ``synthetic_inputs.RangeTheta``."""
    return theta_from_ranges(*rt.astuple())


def matern(nu: float, x: float) -> float:
    return lib().orc_matern(float(nu), float(x))


def cov(theta, h: float, u: float) -> float:
    th = _f64(theta)
    return lib().orc_cov(_d(th), float(h), float(u))


def cov_grad(theta, h: float, u: float) -> np.ndarray:
    th = _f64(theta)
    out = np.zeros(4)
    lib().orc_cov_grad(_d(th), float(h), float(u), _d(out))
    return out


def cov_matrix(xy1, t1, xy2, t2, theta) -> np.ndarray:
    xy1, t1, xy2, t2, th = _f64(xy1), _f64(t1), _f64(xy2), _f64(t2), _f64(theta)
    out = np.zeros((t1.shape[0], t2.shape[0]))
    lib().orc_cov_matrix(t1.shape[0], _d(xy1), _d(t1), t2.shape[0], _d(xy2), _d(t2), _d(th), _d(out))
    return out


def cond_estimates(xy, t, theta, nn, nn_cnt, rows=None) -> np.ndarray:
    """Condition estimate of each row's local block, the quantity the mixed
    form's FP64-fallback rule compares with its threshold (a reading for the
    mixed-precision control, which the paper does not have): the response
    covariance Sigma~ of the positions (N(i) in the order of nn[i], then i)
    with the nugget on the diagonal (Sect. 3.1, Eq. (2)), its Cholesky factor's
    pivots L_jj, and (max_j L_jj / min_j L_jj)^2.  numpy's Cholesky of the
    oracle's covariance matrix; rows with no neighbour give 1."""
    xy, t, th = _f64(xy), _f64(t), _f64(theta)
    rows = np.arange(t.shape[0]) if rows is None else np.asarray(rows)
    out = np.ones(rows.shape[0])
    for q, i in enumerate(rows):
        c = int(nn_cnt[i])
        if c == 0:
            continue
        idx = np.concatenate([np.asarray(nn[i][:c], dtype=np.int64), [i]])
        K = cov_matrix(xy[idx], t[idx], xy[idx], t[idx], th) + th[4] * np.eye(c + 1)
        d = np.diag(np.linalg.cholesky(K))
        out[q] = (d.max() / d.min()) ** 2
    return out


def knn(xy, t, theta, m, rows=None, threads=None):
    """Brute-force correlation neighbours.  Returns (nn int32 [r,m] (-1 pad),
    nn_cnt int32 [r], rho_m [r], rho_m1 [r]) for the requested rows (all by default)."""
    xy, t, th = _f64(xy), _f64(t), _f64(theta)
    n = t.shape[0]
    rows = np.arange(n, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    R = rows.shape[0]
    nn = np.full((R, m), -1, dtype=np.int32)
    cnt = np.zeros(R, dtype=np.int32)
    rm = np.zeros(R)
    rm1 = np.zeros(R)
    lib().orc_knn_rows(n, _d(xy), _d(t), _d(th), int(m), R, rows.ctypes.data_as(_I64),
                       nn.ctypes.data_as(_I32), cnt.ctypes.data_as(_I32), _d(rm), _d(rm1),
                       int(threads or default_threads()))
    return nn, cnt, rm, rm1


class CoverTree:
    """The cover tree of Algorithm 1 (Sect. 4.4.1) over the points in their
    index order, under d_c = sqrt(1 - |rho|); the search of Algorithm 2 by
    knn().  Use as a context manager or call close()."""

    def __init__(self, xy, t, theta):
        self.xy, self.t, self.th = _f64(xy), _f64(t), _f64(theta)
        self.n = self.t.shape[0]
        self.h = lib().orc_cover_tree_build(self.n, _d(self.xy), _d(self.t), _d(self.th))

    @property
    def depth(self) -> int:
        return int(lib().orc_cover_tree_depth(self.h))

    def structure(self):
        """(level [n] int32, parent [n] int64, -1 for the root)."""
        level = np.zeros(self.n, dtype=np.int32)
        parent = np.zeros(self.n, dtype=np.int64)
        lib().orc_cover_tree_structure(self.h, self.n, level.ctypes.data_as(_I32), parent.ctypes.data_as(_I64))
        return level, parent

    def knn(self, m, rows=None, threads=None):
        """As knn() (same outputs, same tie order), by the cover-tree search."""
        rows = np.arange(self.n, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
        R = rows.shape[0]
        nn = np.full((R, m), -1, dtype=np.int32)
        cnt = np.zeros(R, dtype=np.int32)
        rm = np.zeros(R)
        rm1 = np.zeros(R)
        lib().orc_knn_cover_tree(self.h, self.n, _d(self.xy), _d(self.t), _d(self.th), int(m), R,
                                 rows.ctypes.data_as(_I64), nn.ctypes.data_as(_I32), cnt.ctypes.data_as(_I32),
                                 _d(rm), _d(rm1), int(threads or default_threads()))
        return nn, cnt, rm, rm1

    def close(self):
        if getattr(self, "h", None):
            lib().orc_cover_tree_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tie_rows(rho_m, rho_m1, rel: float = 1e-12) -> np.ndarray:
    """Rows whose m-th and (m+1)-th correlations differ by less than rel (relative)."""
    with np.errstate(invalid="ignore"):
        tie = np.isfinite(rho_m) & np.isfinite(rho_m1) & ((rho_m - rho_m1) <= rel * np.abs(rho_m))
    return np.nonzero(tie)[0]


def factor(xy, t, theta, m, nn, nn_cnt, threads=None):
    xy, t, th = _f64(xy), _f64(t), _f64(theta)
    nn, nn_cnt = _i32(nn), _i32(nn_cnt)
    n = t.shape[0]
    A = np.zeros((n, m))
    D = np.zeros(n)
    bad = lib().orc_factor(n, _d(xy), _d(t), _d(th), int(m), nn.ctypes.data_as(_I32),
                           nn_cnt.ctypes.data_as(_I32), _d(A), _d(D), int(threads or default_threads()))
    if bad >= 0:
        raise np.linalg.LinAlgError(f"local block not SPD at row {bad}")
    return A, D


def factor_rows(xy, t, theta, m, rows, nn_rows, cnt_rows, threads=None):
    """A, D of the given rows with the given neighbour lists (spot checks)."""
    xy, t, th = _f64(xy), _f64(t), _f64(theta)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    nn_rows, cnt_rows = _i32(nn_rows), _i32(cnt_rows)
    R = rows.shape[0]
    A = np.zeros((R, m))
    D = np.zeros(R)
    lib().orc_factor_rows(t.shape[0], _d(xy), _d(t), _d(th), int(m), R, rows.ctypes.data_as(_I64),
                          nn_rows.ctypes.data_as(_I32), cnt_rows.ctypes.data_as(_I32), _d(A), _d(D),
                          int(threads or default_threads()))
    return A, D


def nll(xy, t, theta, m, nn, nn_cnt, y, terms=False, threads=None):
    xy, t, th, y = _f64(xy), _f64(t), _f64(theta), _f64(y)
    nn, nn_cnt = _i32(nn), _i32(nn_cnt)
    n = t.shape[0]
    term = np.zeros(n) if terms else None
    v = lib().orc_nll(n, _d(xy), _d(t), _d(th), int(m), nn.ctypes.data_as(_I32), nn_cnt.ctypes.data_as(_I32),
                      _d(y), _d(term) if terms else None, int(threads or default_threads()))
    return (v, term) if terms else v


def nll_grad(xy, t, theta, m, nn, nn_cnt, y, terms=False, threads=None):
    xy, t, th, y = _f64(xy), _f64(t), _f64(theta), _f64(y)
    nn, nn_cnt = _i32(nn), _i32(nn_cnt)
    n = t.shape[0]
    g = np.zeros(5)
    gt = np.zeros((n, 5)) if terms else None
    v = lib().orc_nll_grad(n, _d(xy), _d(t), _d(th), int(m), nn.ctypes.data_as(_I32),
                           nn_cnt.ctypes.data_as(_I32), _d(y), _d(g), _d(gt) if terms else None,
                           int(threads or default_threads()))
    return (v, g, gt) if terms else (v, g)


def nll_grad_rows(xy, t, theta, m, rows, nn_rows, cnt_rows, y, threads=None):
    """Sum of the NLL terms and gradient terms of the given rows (no constant)."""
    xy, t, th, y = _f64(xy), _f64(t), _f64(theta), _f64(y)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    nn_rows, cnt_rows = _i32(nn_rows), _i32(cnt_rows)
    g = np.zeros(5)
    v = lib().orc_nll_grad_rows(t.shape[0], _d(xy), _d(t), _d(th), int(m), rows.shape[0],
                                rows.ctypes.data_as(_I64), nn_rows.ctypes.data_as(_I32),
                                cnt_rows.ctypes.data_as(_I32), _d(y), _d(g), int(threads or default_threads()))
    return v, g


def vecchia_sample(m, nn, nn_cnt, A, D, z):
    nn, nn_cnt, A, D, z = _i32(nn), _i32(nn_cnt), _f64(A), _f64(D), _f64(z)
    y = np.zeros(z.shape[0])
    lib().orc_vecchia_sample(z.shape[0], int(m), nn.ctypes.data_as(_I32), nn_cnt.ctypes.data_as(_I32),
                             _d(A), _d(D), _d(z), _d(y))
    return y


def dense_nll(xy, t, theta, y, grad=False):
    xy, t, th, y = _f64(xy), _f64(t), _f64(theta), _f64(y)
    g = np.zeros(5)
    v = lib().orc_dense_nll(t.shape[0], _d(xy), _d(t), _d(th), _d(y), _d(g) if grad else None)
    return (v, g) if grad else v


def dense_sample(xy, t, theta, z):
    xy, t, th, z = _f64(xy), _f64(t), _f64(theta), _f64(z)
    y = np.zeros(z.shape[0])
    if lib().orc_dense_sample(t.shape[0], _d(xy), _d(t), _d(th), _d(z), _d(y)) != 0:
        raise np.linalg.LinAlgError("covariance not SPD")
    return y


def all_predecessors(n: int):
    """Neighbour sets N(i) = {0..i-1} (m = n-1): the exact factorisation."""
    m = max(n - 1, 1)
    nn = np.full((n, m), -1, dtype=np.int32)
    for i in range(1, n):
        nn[i, :i] = np.arange(i, dtype=np.int32)
    cnt = np.minimum(np.arange(n), m).astype(np.int32)
    return m, nn, cnt
