"""GB300 (sm_103a) Vecchia / VIF space-time likelihood engine.

Python binding of ``libvst.so`` (C ABI in ``include/vst.h``).  The functions
here carry the C entry points' names and only marshal arguments: every step
of the computation runs in the library's CUDA kernels.  PyTorch supplies
device memory (CUDA tensors), streams, and the autograd wrapper.

There is no CPU path: loading fails loudly if ``libvst.so`` is missing (run
``python -m paper_2602_03609_gb300.build`` or ``__graft_entry__.build()``).

Layouts (row i of every array is point i in Vecchia order):
    xy  float64 [n, 2]     t  float64 [n]     y  float64 [n]
    nn  int32 [n, m] (-1 padded)              nn_cnt  int32 [n]
    A   float64 [n, m]  (B[i, nn[i, q]] = -A[i, q])   D  float64 [n]
theta: native parameters of Eq. (2) as a sequence
    (sigma1sq, c, a, gamma, nugget, alpha, delta, nu)
gradients are with respect to (sigma1sq, c, a, gamma, nugget).
"""
from __future__ import annotations

import ctypes
import os

import torch

__all__ = [
    "FP64", "MIXED", "MAX_M", "VstError", "lib", "vst_theta_from_ranges", "vst_workspace_size",
    "vst_workspace_size_vif_grad",
    "Workspace", "vif_build_neighbors", "vecchia_factor", "vecchia_nll", "vecchia_nll_grad",
    "vecchia_sample", "vst_workspace_status", "VecchiaNLL", "theta_tuple", "vst_profile_enable",
    "vst_profile_read", "vecchia_nll_grad_noalloc", "vst_noalloc_status", "NOALLOC_MAX_N",
    "BatchedWorkspace", "vecchia_nll_grad_batched", "BatchedGraph", "vst_autotune_nll_grad",
    "vst_autotune_nll_grad_batched", "vst_autotune_clear", "MIXED_BF16X3", "vif_lowrank_u", "vif_gram_tc",
    "vst_workspace_size_gram_tc",
    "vecchia_predict", "vst_workspace_size_predict", "PredictWorkspace", "sts_kmeanspp",
    "vecchia_nll_grad_ex", "vecchia_nll_grad_batched_ex", "vecchia_sample_ex", "vst_noalloc_scratch_bytes",
]

FP64 = 0
MIXED = 1
MIXED_BF16X3 = 2
MAX_M = 31
_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvst.so")

_STATUS = {0: "VST_OK", 1: "VST_EINVAL", 2: "VST_ENOMEM", 3: "VST_ENOTSPD", 4: "VST_ETIMEOUT",
           5: "VST_ECUDA", 6: "VST_EINTERNAL"}


class VstError(RuntimeError):
    def __init__(self, code, msg, info=None):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code
        self.info = info


class _Theta(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("sigma1sq", "c", "a", "gamma", "nugget", "alpha", "delta", "nu")]


class _Points(ctypes.Structure):
    _fields_ = [("xy", ctypes.c_void_p), ("t", ctypes.c_void_p), ("n", ctypes.c_int64)]


class _Inducing(ctypes.Structure):
    _fields_ = [("xy", ctypes.c_void_p), ("t", ctypes.c_void_p), ("k", ctypes.c_int64)]


class WsInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_int32), ("bad_row", ctypes.c_int64),
                ("n_fallback", ctypes.c_int64), ("n_tie", ctypes.c_int64)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class _Options(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("row_begin", ctypes.c_int64), ("row_end", ctypes.c_int64),
                ("fallback_rows", ctypes.c_void_p), ("wait_limit", ctypes.c_int64)]


class TuneResult(ctypes.Structure):
    _fields_ = [("blocks_per_sm", ctypes.c_int), ("row_chunk", ctypes.c_int), ("ms", ctypes.c_float)]


_lib = None
_P = ctypes.c_void_p


def lib():
    """The loaded libvst.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: the CUDA library must be built "
                              "(python -m paper_2602_03609_gb300.build); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        L.vst_last_error.restype = ctypes.c_char_p
        L.vst_version.restype = ctypes.c_int
        L.vst_theta_from_ranges.restype = ctypes.c_int
        L.vst_theta_from_ranges.argtypes = [ctypes.c_double] * 8 + [ctypes.POINTER(_Theta)]
        L.vst_workspace_size.restype = ctypes.c_size_t
        L.vst_workspace_size.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int64]
        L.vst_workspace_size_vif_grad.restype = ctypes.c_size_t
        L.vst_workspace_size_vif_grad.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int64]
        PT, TH, IN = ctypes.POINTER(_Points), ctypes.POINTER(_Theta), ctypes.POINTER(_Inducing)
        L.vif_build_neighbors.restype = ctypes.c_int
        L.vif_build_neighbors.argtypes = [PT, TH, ctypes.c_int, IN, _P, _P, _P, ctypes.c_int64, _P,
                                          ctypes.c_size_t, _P]
        L.vecchia_factor.restype = ctypes.c_int
        L.vecchia_factor.argtypes = [PT, TH, ctypes.c_int, IN, _P, _P, ctypes.c_int, _P, _P, _P,
                                     ctypes.c_size_t, _P]
        L.vecchia_nll.restype = ctypes.c_int
        L.vecchia_nll.argtypes = [PT, TH, ctypes.c_int, IN, _P, _P, _P, ctypes.c_int, _P, _P, ctypes.c_size_t, _P]
        L.vecchia_nll_grad.restype = ctypes.c_int
        L.vecchia_nll_grad.argtypes = [PT, TH, ctypes.c_int, IN, _P, _P, _P, ctypes.c_int, _P, _P, _P,
                                       ctypes.c_size_t, _P]
        OP = ctypes.POINTER(_Options)
        L.vecchia_nll_grad_ex.restype = ctypes.c_int
        L.vecchia_nll_grad_ex.argtypes = [PT, TH, ctypes.c_int, IN, _P, _P, _P, ctypes.c_int, OP, _P, _P, _P,
                                          ctypes.c_size_t, _P]
        L.vecchia_sample_ex.restype = ctypes.c_int
        L.vecchia_sample_ex.argtypes = [PT, TH, ctypes.c_int, _P, _P, _P, _P, OP, _P, ctypes.c_size_t, _P]
        L.vst_workspace_size_kmeans.restype = ctypes.c_size_t
        L.vst_workspace_size_kmeans.argtypes = [ctypes.c_int64]
        L.vst_sts_kmeanspp.restype = ctypes.c_int
        L.vst_sts_kmeanspp.argtypes = [PT, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, _P, _P, ctypes.c_int64,
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64), _P, ctypes.c_size_t, _P]
        L.vst_workspace_size_predict.restype = ctypes.c_size_t
        L.vst_workspace_size_predict.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
        L.vecchia_predict.restype = ctypes.c_int
        L.vecchia_predict.argtypes = [PT, TH, ctypes.c_int, _P, PT, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P,
                                      ctypes.c_size_t, _P]
        L.vif_lowrank_u.restype = ctypes.c_int
        L.vif_lowrank_u.argtypes = [PT, TH, IN, ctypes.c_int, _P, _P, _P, ctypes.c_size_t, _P]
        L.vst_workspace_size_gram_tc.restype = ctypes.c_size_t
        L.vst_workspace_size_gram_tc.argtypes = [ctypes.c_int64, ctypes.c_int]
        L.vif_gram_tc.restype = ctypes.c_int
        L.vif_gram_tc.argtypes = [ctypes.c_int64, ctypes.c_int, _P, ctypes.c_int64, _P, ctypes.c_int64, _P, _P,
                                  ctypes.c_size_t, _P]
        L.vecchia_sample.restype = ctypes.c_int
        L.vecchia_sample.argtypes = [PT, TH, ctypes.c_int, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]
        L.vst_profile_enable.restype = None
        L.vst_profile_enable.argtypes = [ctypes.c_int]
        L.vst_profile_read.restype = ctypes.c_int
        L.vst_profile_read.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
        L.vecchia_nll_grad_noalloc.restype = ctypes.c_int
        L.vecchia_nll_grad_noalloc.argtypes = [PT, TH, ctypes.c_int, _P, _P, _P, ctypes.c_int, _P, _P, _P]
        L.vst_noalloc_scratch_bytes.restype = ctypes.c_size_t
        L.vst_noalloc_scratch_bytes.argtypes = []
        L.vst_noalloc_status.restype = ctypes.c_int
        L.vst_noalloc_status.argtypes = [_P, ctypes.POINTER(WsInfo)]
        I64 = ctypes.c_int64
        L.vst_workspace_size_batched.restype = ctypes.c_size_t
        L.vst_workspace_size_batched.argtypes = [ctypes.c_int, I64, ctypes.c_int]
        bargs = [ctypes.c_int, I64, _P, _P, ctypes.c_double, _P, _P, ctypes.c_int, _P, _P, _P, ctypes.c_int, _P, _P,
                 _P, ctypes.c_size_t]
        L.vecchia_nll_grad_batched.restype = ctypes.c_int
        L.vecchia_nll_grad_batched.argtypes = bargs + [_P]
        L.vecchia_nll_grad_batched_ex.restype = ctypes.c_int
        L.vecchia_nll_grad_batched_ex.argtypes = bargs[:12] + [OP] + bargs[12:] + [_P]
        L.vst_graph_capture_nll_grad_batched.restype = ctypes.c_int
        L.vst_graph_capture_nll_grad_batched.argtypes = bargs + [ctypes.POINTER(ctypes.c_void_p)]
        L.vst_graph_launch.restype = ctypes.c_int
        L.vst_graph_launch.argtypes = [_P, _P]
        L.vst_graph_destroy.restype = ctypes.c_int
        L.vst_graph_destroy.argtypes = [_P]
        L.vst_autotune_nll_grad.restype = ctypes.c_int
        L.vst_autotune_nll_grad.argtypes = [PT, TH, ctypes.c_int, _P, _P, _P, ctypes.c_int, _P, ctypes.c_size_t, _P,
                                            ctypes.POINTER(TuneResult)]
        L.vst_autotune_nll_grad_batched.restype = ctypes.c_int
        L.vst_autotune_nll_grad_batched.argtypes = bargs + [_P, ctypes.POINTER(TuneResult)]
        L.vst_autotune_clear.restype = None
        L.vst_autotune_clear.argtypes = []
        L.vst_workspace_status.restype = ctypes.c_int
        L.vst_workspace_status.argtypes = [_P, _P, ctypes.POINTER(WsInfo)]
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise VstError(rc, lib().vst_last_error().decode())


def theta_tuple(theta):
    if isinstance(theta, _Theta):
        return tuple(getattr(theta, k) for k, _ in _Theta._fields_)
    t = tuple(float(v) for v in (theta.tolist() if hasattr(theta, "tolist") else theta))
    if len(t) != 8:
        raise ValueError("theta needs 8 values (sigma1sq, c, a, gamma, nugget, alpha, delta, nu)")
    return t


def _th(theta):
    return _Theta(*theta_tuple(theta))


def vst_theta_from_ranges(sigma1sq, range_s, range_t, gamma, nugget, alpha=0.4, delta=0.2, nu=1.5):
    out = _Theta()
    _check(lib().vst_theta_from_ranges(sigma1sq, range_s, range_t, gamma, nugget, alpha, delta, nu,
                                       ctypes.byref(out)))
    return theta_tuple(out)


def vst_workspace_size(n, m, k=0) -> int:
    return int(lib().vst_workspace_size(int(n), int(m), int(k)))


def vst_workspace_size_vif_grad(n, m, k) -> int:
    return int(lib().vst_workspace_size_vif_grad(int(n), int(m), int(k)))


class Workspace:
    """Caller-owned scratch memory (a CUDA uint8 tensor, 256-byte aligned).
    vif_grad=True sizes it for the VIF gradient (k > 0)."""

    def __init__(self, n, m, k=0, device=None, vif_grad=False):
        self.nbytes = vst_workspace_size_vif_grad(n, m, k) if (vif_grad and k > 0) else vst_workspace_size(n, m, k)
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device or "cuda")
        self.ptr = (self.buf.data_ptr() + 255) // 256 * 256

    def fits(self, n, m, k=0, vif_grad=False):
        need = vst_workspace_size_vif_grad(n, m, k) if (vif_grad and k > 0) else vst_workspace_size(n, m, k)
        return self.nbytes >= need


def _ptr(x, dtype, name):
    if x is None:
        return None
    if not (isinstance(x, torch.Tensor) and x.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return x.data_ptr()


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _points(xy, t):
    n = t.shape[0]
    if xy.shape != (n, 2):
        raise ValueError("xy must be [n, 2]")
    return _Points(_ptr(xy, torch.float64, "xy"), _ptr(t, torch.float64, "t"), n)


def _ws(ws, n, m, k=0, vif_grad=False):
    if ws is None:
        ws = Workspace(n, m, k, vif_grad=vif_grad)
    if not ws.fits(n, m, k, vif_grad=vif_grad):
        raise ValueError("workspace too small")
    return ws


def _inducing(inducing):
    """(xyk [k,2], tk [k]) CUDA float64 tensors, or None for plain Vecchia."""
    if inducing is None:
        return None, 0
    xyk, tk = inducing
    k = tk.shape[0]
    if xyk.shape != (k, 2):
        raise ValueError("inducing xy must be [k, 2]")
    return _Inducing(_ptr(xyk, torch.float64, "inducing xy"), _ptr(tk, torch.float64, "inducing t"), k), k


def vif_build_neighbors(xy, t, theta, m, nn=None, nn_cnt=None, tie_rows=None, ws=None, stream=None, inducing=None):
    """Correlation-based neighbour sets (Sect. 4.4.1); with inducing=(xyk, tk),
    by the VIF residual correlation (Sect. 4.3).  Returns (nn, nn_cnt)."""
    n = t.shape[0]
    ind, k = _inducing(inducing)
    nn = nn if nn is not None else torch.empty((n, m), dtype=torch.int32, device=t.device)
    nn_cnt = nn_cnt if nn_cnt is not None else torch.empty(n, dtype=torch.int32, device=t.device)
    ws = _ws(ws, n, m, k)
    pts = _points(xy, t)
    cap = 0 if tie_rows is None else tie_rows.numel()
    _check(lib().vif_build_neighbors(ctypes.byref(pts), ctypes.byref(_th(theta)), int(m),
                                     ctypes.byref(ind) if ind else None,
                                     _ptr(nn, torch.int32, "nn"), _ptr(nn_cnt, torch.int32, "nn_cnt"),
                                     _ptr(tie_rows, torch.int64, "tie_rows"), cap, ws.ptr, ws.nbytes,
                                     _stream(stream)))
    return nn, nn_cnt


def vecchia_factor(xy, t, theta, m, nn, nn_cnt, precision=FP64, A=None, D=None, ws=None, stream=None,
                   inducing=None):
    """Vecchia factor (A, D) of the response covariance (Sect. 4.1), or of the
    VIF residual with inducing=(xyk, tk) (Sect. 4.3)."""
    n = t.shape[0]
    ind, k = _inducing(inducing)
    A = A if A is not None else torch.empty((n, m), dtype=torch.float64, device=t.device)
    D = D if D is not None else torch.empty(n, dtype=torch.float64, device=t.device)
    ws = _ws(ws, n, m, k)
    pts = _points(xy, t)
    _check(lib().vecchia_factor(ctypes.byref(pts), ctypes.byref(_th(theta)), int(m), ctypes.byref(ind) if ind else None,
                                _ptr(nn, torch.int32, "nn"), _ptr(nn_cnt, torch.int32, "nn_cnt"), int(precision),
                                _ptr(A, torch.float64, "A"), _ptr(D, torch.float64, "D"), ws.ptr, ws.nbytes,
                                _stream(stream)))
    return A, D


def vecchia_nll(xy, t, theta, m, nn, nn_cnt, y, precision=FP64, out=None, ws=None, stream=None, inducing=None):
    """Vecchia (or, with inducing=(xyk, tk), VIF) negative log-likelihood;
    returns a 1-element CUDA float64 tensor."""
    n = t.shape[0]
    ind, k = _inducing(inducing)
    out = out if out is not None else torch.empty(1, dtype=torch.float64, device=t.device)
    ws = _ws(ws, n, m, k)
    pts = _points(xy, t)
    _check(lib().vecchia_nll(ctypes.byref(pts), ctypes.byref(_th(theta)), int(m), ctypes.byref(ind) if ind else None,
                             _ptr(nn, torch.int32, "nn"), _ptr(nn_cnt, torch.int32, "nn_cnt"),
                             _ptr(y, torch.float64, "y"), int(precision), _ptr(out, torch.float64, "nll"),
                             ws.ptr, ws.nbytes, _stream(stream)))
    return out


def vecchia_nll_grad(xy, t, theta, m, nn, nn_cnt, y, precision=FP64, nll=None, grad=None, ws=None, stream=None,
                     inducing=None):
    """NLL and its gradient w.r.t. (sigma1sq, c, a, gamma, nugget); CUDA tensors.
    With inducing=(xyk, tk): the VIF likelihood (Sect. 4.3), FP64 or mixed
    (a workspace passed in must then be sized with vif_grad=True)."""
    n = t.shape[0]
    ind, k = _inducing(inducing)
    nll = nll if nll is not None else torch.empty(1, dtype=torch.float64, device=t.device)
    grad = grad if grad is not None else torch.empty(5, dtype=torch.float64, device=t.device)
    ws = _ws(ws, n, m, k, vif_grad=True)
    pts = _points(xy, t)
    _check(lib().vecchia_nll_grad(ctypes.byref(pts), ctypes.byref(_th(theta)), int(m),
                                  ctypes.byref(ind) if ind else None,
                                  _ptr(nn, torch.int32, "nn"), _ptr(nn_cnt, torch.int32, "nn_cnt"),
                                  _ptr(y, torch.float64, "y"), int(precision), _ptr(nll, torch.float64, "nll"),
                                  _ptr(grad, torch.float64, "grad"), ws.ptr, ws.nbytes, _stream(stream)))
    return nll, grad


def _options(tau=0.0, row_begin=0, row_end=0, fallback_rows=None, wait_limit=0):
    return _Options(float(tau), int(row_begin), int(row_end), _ptr(fallback_rows, torch.uint8, "fallback_rows"),
                    int(wait_limit))


def vecchia_nll_grad_ex(xy, t, theta, m, nn, nn_cnt, y, precision=FP64, tau=0.0, row_begin=0, row_end=0,
                        fallback_rows=None, nll=None, grad=None, ws=None, stream=None):
    """vecchia_nll_grad (plain Vecchia) with options: tau (the mixed form's
    condition threshold, 0 = default 1e4), the row range [row_begin, row_end)
    (row_end = 0: n) and fallback_rows (a CUDA uint8 [n] tensor receiving 1 for
    each row redone in FP64)."""
    n = t.shape[0]
    nll = nll if nll is not None else torch.empty(1, dtype=torch.float64, device=t.device)
    grad = grad if grad is not None else torch.empty(5, dtype=torch.float64, device=t.device)
    ws = _ws(ws, n, m)
    pts = _points(xy, t)
    opt = _options(tau, row_begin, row_end, fallback_rows)
    _check(lib().vecchia_nll_grad_ex(ctypes.byref(pts), ctypes.byref(_th(theta)), int(m), None,
                                     _ptr(nn, torch.int32, "nn"), _ptr(nn_cnt, torch.int32, "nn_cnt"),
                                     _ptr(y, torch.float64, "y"), int(precision), ctypes.byref(opt),
                                     _ptr(nll, torch.float64, "nll"), _ptr(grad, torch.float64, "grad"), ws.ptr,
                                     ws.nbytes, _stream(stream)))
    return nll, grad


def vif_lowrank_u(xy, t, theta, inducing, precision=FP64, U=None, r=None, ws=None, stream=None):
    """VIF low rank (Sect. 4.3): U = Sigma_nk L^{-T} [n, k] and the residual
    variances r = sigma1sq - ||U_i||^2 [n]; CUDA float64 tensors."""
    n = t.shape[0]
    ind, k = _inducing(inducing)
    if ind is None:
        raise ValueError("vif_lowrank_u needs inducing=(xyk, tk) with k > 0")
    U = U if U is not None else torch.empty((n, k), dtype=torch.float64, device=t.device)
    r = r if r is not None else torch.empty(n, dtype=torch.float64, device=t.device)
    ws = _ws(ws, n, 0, k)
    pts = _points(xy, t)
    _check(lib().vif_lowrank_u(ctypes.byref(pts), ctypes.byref(_th(theta)), ctypes.byref(ind), int(precision),
                               _ptr(U, torch.float64, "U"), _ptr(r, torch.float64, "r"), ws.ptr, ws.nbytes,
                               _stream(stream)))
    return U, r


def vst_workspace_size_gram_tc(n, kc) -> int:
    return int(lib().vst_workspace_size_gram_tc(int(n), int(kc)))


def _rows_f32(x, name, kc):
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32 and x.dim() == 2):
        raise TypeError(f"{name} must be a 2-D CUDA float32 tensor")
    if x.shape[1] != kc or x.stride(1) != 1 or (x.shape[0] > 1 and x.stride(0) < kc):
        raise ValueError(f"{name} must be [n, kc] with unit column stride")
    return x.data_ptr(), max(int(x.stride(0)), kc)


def vif_gram_tc(A, B=None, C=None, ws=None, stream=None):
    """C = A^T B (A^T A when B is None), [kc, kc] float64, on the tensor cores
    with the fixed-point BF16 split, exponents per column and 128-row block
    (the contraction over the points of the VIF's Woodbury form, Sect. 4.3).  A, B: [n, kc] CUDA float32 tensors whose
    rows may be strided.  ws: a CUDA uint8 tensor of at least
    vst_workspace_size_gram_tc(n, kc) bytes (allocated when None); its status
    header is read by vst_workspace_status(ws)."""
    n, kc = A.shape
    pa, lda = _rows_f32(A, "A", kc)
    pb, ldb = (None, 0) if B is None else _rows_f32(B, "B", kc)
    if B is not None and B.shape[0] != n:
        raise ValueError("A and B need the same number of rows")
    C = C if C is not None else torch.empty((kc, kc), dtype=torch.float64, device=A.device)
    need = vst_workspace_size_gram_tc(n, kc)
    if ws is None:
        ws = _RawWorkspace(need, A.device)
    if ws.nbytes < need:
        raise ValueError("workspace too small")
    _check(lib().vif_gram_tc(int(n), int(kc), pa, lda, pb, ldb, _ptr(C, torch.float64, "C"), ws.ptr, ws.nbytes,
                             _stream(stream)))
    return C


class _RawWorkspace(Workspace):
    """A workspace of a given byte count (vif_gram_tc)."""

    def __init__(self, nbytes, device=None):
        self.nbytes = int(nbytes)
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device or "cuda")
        self.ptr = (self.buf.data_ptr() + 255) // 256 * 256


def vst_workspace_size_predict(n_train, n_pred, m) -> int:
    return int(lib().vst_workspace_size_predict(int(n_train), int(n_pred), int(m)))


class PredictWorkspace(Workspace):
    """Workspace of vecchia_predict."""

    def __init__(self, n_train, n_pred, m, device=None):
        self.nbytes = vst_workspace_size_predict(n_train, n_pred, m)
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device or "cuda")
        self.ptr = (self.buf.data_ptr() + 255) // 256 * 256

    def fits(self, n_train, n_pred, m):
        return self.nbytes >= vst_workspace_size_predict(n_train, n_pred, m)


def vecchia_predict(xy, t, y, theta, m, xy_pred, t_pred, precision=FP64, latent=False, mean=None, var=None,
                    nn=None, ws=None, stream=None):
    """Vecchia predictive mean and variance at new points (each conditioned on
    its m most correlated training points).  Returns (mean, var), or
    (mean, var, nn) when nn=True (the neighbour indices, [n_pred, m] int32)."""
    n, npred = t.shape[0], t_pred.shape[0]
    mean = mean if mean is not None else torch.empty(npred, dtype=torch.float64, device=t_pred.device)
    var = var if var is not None else torch.empty(npred, dtype=torch.float64, device=t_pred.device)
    want_nn = nn is True
    if want_nn:
        nn = torch.empty((npred, m), dtype=torch.int32, device=t_pred.device)
    if ws is None:
        ws = PredictWorkspace(n, npred, m, device=t_pred.device)
    if not ws.fits(n, npred, m):
        raise ValueError("workspace too small")
    tr, pr = _points(xy, t), _points(xy_pred, t_pred)
    _check(lib().vecchia_predict(ctypes.byref(tr), ctypes.byref(_th(theta)), int(m), _ptr(y, torch.float64, "y"),
                                 ctypes.byref(pr), int(precision), 1 if latent else 0,
                                 _ptr(mean, torch.float64, "mean"), _ptr(var, torch.float64, "var"),
                                 _ptr(nn, torch.int32, "nn") if want_nn else None, ws.ptr, ws.nbytes,
                                 _stream(stream)))
    return (mean, var, nn) if want_nn else (mean, var)


def sts_kmeanspp(xy, t, m, seed=0, lloyd_iters=10, k_cap=None, stream=None):
    """Space-time separated kMeans++ inducing points (Algorithm 3).  Returns
    (xyk [k, 2], tk [k]) CUDA float64 tensors and (m_s, m_t)."""
    n = t.shape[0]
    k_cap = int(k_cap if k_cap is not None else 4 * m + 16)
    xyk = torch.empty((k_cap, 2), dtype=torch.float64, device=t.device)
    tk = torch.empty(k_cap, dtype=torch.float64, device=t.device)
    nbytes = int(lib().vst_workspace_size_kmeans(int(n)))
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=t.device)
    ptr = (buf.data_ptr() + 255) // 256 * 256
    k, ms, mt = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    pts = _points(xy, t)
    _check(lib().vst_sts_kmeanspp(ctypes.byref(pts), int(m), ctypes.c_uint64(seed & (2**64 - 1)), int(lloyd_iters),
                                  xyk.data_ptr(), tk.data_ptr(), k_cap, ctypes.byref(k), ctypes.byref(ms),
                                  ctypes.byref(mt), ptr, nbytes, _stream(stream)))
    return xyk[:k.value], tk[:k.value], (ms.value, mt.value)


class BatchedWorkspace(Workspace):
    """Workspace of the batched entry points."""

    def __init__(self, nsets, n_total, m, device=None):
        self.nbytes = int(lib().vst_workspace_size_batched(int(nsets), int(n_total), int(m)))
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device or "cuda")
        self.ptr = (self.buf.data_ptr() + 255) // 256 * 256

    def fits(self, nsets, n_total, m):
        return self.nbytes >= int(lib().vst_workspace_size_batched(int(nsets), int(n_total), int(m)))


def _batched_args(offsets, thetas, nu, xy, t, m, nn, nn_cnt, y, precision, nll, grad, ws):
    nsets = offsets.numel() - 1
    n = t.shape[0]
    if thetas.shape != (nsets, 8):
        raise ValueError("thetas must be a CUDA float64 tensor [nsets, 8] "
                         "(sigma1sq, c, a, gamma, nugget, alpha, delta, nu)")
    if xy.shape != (n, 2):
        raise ValueError("xy must be [n, 2]")
    if not ws.fits(nsets, n, m):
        raise ValueError("workspace too small")
    return [nsets, n, _ptr(offsets, torch.int64, "offsets"), _ptr(thetas, torch.float64, "thetas"), float(nu),
            _ptr(xy, torch.float64, "xy"), _ptr(t, torch.float64, "t"), int(m), _ptr(nn, torch.int32, "nn"),
            _ptr(nn_cnt, torch.int32, "nn_cnt"), _ptr(y, torch.float64, "y"), int(precision),
            _ptr(nll, torch.float64, "nll"), _ptr(grad, torch.float64, "grad"), ws.ptr, ws.nbytes]


def vecchia_nll_grad_batched(offsets, thetas, nu, xy, t, m, nn, nn_cnt, y, precision=FP64, nll=None, grad=None,
                             ws=None, stream=None):
    """NLL [nsets] and gradient [nsets, 5] of independent datasets in one launch.
    offsets: CUDA int64 [nsets+1]; thetas: CUDA float64 [nsets, 8]; neighbour
    indices local to each dataset."""
    nsets = offsets.numel() - 1
    nll = nll if nll is not None else torch.empty(nsets, dtype=torch.float64, device=t.device)
    grad = grad if grad is not None else torch.empty((nsets, 5), dtype=torch.float64, device=t.device)
    ws = ws if ws is not None else BatchedWorkspace(nsets, t.shape[0], m)
    args = _batched_args(offsets, thetas, nu, xy, t, m, nn, nn_cnt, y, precision, nll, grad, ws)
    _check(lib().vecchia_nll_grad_batched(*args, _stream(stream)))
    return nll, grad


def vecchia_nll_grad_batched_ex(offsets, thetas, nu, xy, t, m, nn, nn_cnt, y, precision=FP64, tau=0.0,
                                fallback_rows=None, nll=None, grad=None, ws=None, stream=None):
    """vecchia_nll_grad_batched with options: tau and fallback_rows (CUDA uint8
    [n_total])."""
    nsets = offsets.numel() - 1
    nll = nll if nll is not None else torch.empty(nsets, dtype=torch.float64, device=t.device)
    grad = grad if grad is not None else torch.empty((nsets, 5), dtype=torch.float64, device=t.device)
    ws = ws if ws is not None else BatchedWorkspace(nsets, t.shape[0], m)
    args = _batched_args(offsets, thetas, nu, xy, t, m, nn, nn_cnt, y, precision, nll, grad, ws)
    opt = _options(tau, 0, 0, fallback_rows)
    _check(lib().vecchia_nll_grad_batched_ex(*args[:12], ctypes.byref(opt), *args[12:], _stream(stream)))
    return nll, grad


class BatchedGraph:
    """A captured CUDA graph of one batched evaluation (vst_graph_*)."""

    def __init__(self, offsets, thetas, nu, xy, t, m, nn, nn_cnt, y, precision, nll, grad, ws):
        self._keep = (offsets, thetas, xy, t, nn, nn_cnt, y, nll, grad, ws)
        self.nll, self.grad = nll, grad
        h = ctypes.c_void_p(None)
        args = _batched_args(offsets, thetas, nu, xy, t, m, nn, nn_cnt, y, precision, nll, grad, ws)
        _check(lib().vst_graph_capture_nll_grad_batched(*args, ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(lib().vst_graph_launch(self._h, _stream(stream)))
        return self.nll, self.grad

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().vst_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vst_autotune_nll_grad(xy, t, theta, m, nn, nn_cnt, y, precision=MIXED, ws=None, stream=None):
    """Pick and cache the fastest launch shape; returns (blocks_per_sm, row_chunk, ms)."""
    n = t.shape[0]
    ws = _ws(ws, n, m)
    pts = _points(xy, t)
    r = TuneResult()
    _check(lib().vst_autotune_nll_grad(ctypes.byref(pts), ctypes.byref(_th(theta)), int(m),
                                       _ptr(nn, torch.int32, "nn"), _ptr(nn_cnt, torch.int32, "nn_cnt"),
                                       _ptr(y, torch.float64, "y"), int(precision), ws.ptr, ws.nbytes,
                                       _stream(stream), ctypes.byref(r)))
    return r.blocks_per_sm, r.row_chunk, r.ms


def vst_autotune_nll_grad_batched(offsets, thetas, nu, xy, t, m, nn, nn_cnt, y, precision=MIXED, nll=None,
                                  grad=None, ws=None, stream=None):
    nsets = offsets.numel() - 1
    nll = nll if nll is not None else torch.empty(nsets, dtype=torch.float64, device=t.device)
    grad = grad if grad is not None else torch.empty((nsets, 5), dtype=torch.float64, device=t.device)
    ws = ws if ws is not None else BatchedWorkspace(nsets, t.shape[0], m)
    args = _batched_args(offsets, thetas, nu, xy, t, m, nn, nn_cnt, y, precision, nll, grad, ws)
    r = TuneResult()
    _check(lib().vst_autotune_nll_grad_batched(*args, _stream(stream), ctypes.byref(r)))
    return r.blocks_per_sm, r.row_chunk, r.ms


def vst_autotune_clear():
    lib().vst_autotune_clear()


NOALLOC_MAX_N = 1 << 21


def vecchia_nll_grad_noalloc(xy, t, theta, m, nn, nn_cnt, y, precision=FP64, nll=None, grad=None, stream=None):
    """vecchia_nll_grad without a workspace, for callers that cannot allocate
    device memory (the library's own static device scratch of about 74 MiB,
    vst_noalloc_scratch_bytes(), is used; plain Vecchia only; n <=
    NOALLOC_MAX_N; calls that overlap on the GPU race on that scratch).
    nll/grad, if given, must be preallocated CUDA float64 tensors."""
    n = t.shape[0]
    nll = nll if nll is not None else torch.empty(1, dtype=torch.float64, device=t.device)
    grad = grad if grad is not None else torch.empty(5, dtype=torch.float64, device=t.device)
    pts = _points(xy, t)
    _check(lib().vecchia_nll_grad_noalloc(ctypes.byref(pts), ctypes.byref(_th(theta)), int(m),
                                          _ptr(nn, torch.int32, "nn"), _ptr(nn_cnt, torch.int32, "nn_cnt"),
                                          _ptr(y, torch.float64, "y"), int(precision),
                                          _ptr(nll, torch.float64, "nll"), _ptr(grad, torch.float64, "grad"),
                                          _stream(stream)))
    return nll, grad


def vst_noalloc_status(stream=None, raise_on_error=True):
    """Device-side status of the last no-allocation call on the current device."""
    info = WsInfo()
    rc = lib().vst_noalloc_status(_stream(stream), ctypes.byref(info))
    if rc != 0 and raise_on_error:
        raise VstError(rc, lib().vst_last_error().decode(), info.asdict())
    return info.asdict()


def vecchia_sample(xy, t, theta, m, nn, nn_cnt, z, y=None, ws=None, stream=None):
    """y = B^{-1} D^{1/2} z with the FP64 Vecchia factor."""
    n = t.shape[0]
    y = y if y is not None else torch.empty(n, dtype=torch.float64, device=t.device)
    ws = _ws(ws, n, m)
    pts = _points(xy, t)
    _check(lib().vecchia_sample(ctypes.byref(pts), ctypes.byref(_th(theta)), int(m), _ptr(nn, torch.int32, "nn"),
                                _ptr(nn_cnt, torch.int32, "nn_cnt"), _ptr(z, torch.float64, "z"),
                                _ptr(y, torch.float64, "y"), ws.ptr, ws.nbytes, _stream(stream)))
    return y


def vecchia_sample_ex(xy, t, theta, m, nn, nn_cnt, z, wait_limit=0, y=None, ws=None, stream=None):
    """vecchia_sample with a limit on the polls of its bounded device waits
    (wait_limit; 0 = the default of about one second)."""
    n = t.shape[0]
    y = y if y is not None else torch.empty(n, dtype=torch.float64, device=t.device)
    ws = _ws(ws, n, m)
    pts = _points(xy, t)
    opt = _options(wait_limit=wait_limit)
    _check(lib().vecchia_sample_ex(ctypes.byref(pts), ctypes.byref(_th(theta)), int(m), _ptr(nn, torch.int32, "nn"),
                                   _ptr(nn_cnt, torch.int32, "nn_cnt"), _ptr(z, torch.float64, "z"),
                                   _ptr(y, torch.float64, "y"), ctypes.byref(opt), ws.ptr, ws.nbytes,
                                   _stream(stream)))
    return y


def vst_noalloc_scratch_bytes() -> int:
    """Size of the static device scratch of vecchia_nll_grad_noalloc."""
    return int(lib().vst_noalloc_scratch_bytes())


def vst_workspace_status(ws, stream=None, raise_on_error=True):
    """Synchronise and read the device-side status/counters of the last call."""
    info = WsInfo()
    rc = lib().vst_workspace_status(ws.ptr, _stream(stream), ctypes.byref(info))
    if rc != 0 and raise_on_error:
        raise VstError(rc, lib().vst_last_error().decode(), info.asdict())
    return info.asdict()


PROF_ROWS, PROF_FALLBACK, PROF_KNN, PROF_SAMPLE = 0, 1, 2, 3
PROF_VIF_GEMM, PROF_VIF_GRAM, PROF_VIF_SYRK, PROF_VIF_FILTER = 4, 5, 6, 7


def vst_profile_enable(on=True):
    lib().vst_profile_enable(1 if on else 0)


def vst_profile_read(kernel_class):
    """(launches, total device ms) of one kernel class since the last enable."""
    n = ctypes.c_int64(0)
    ms = ctypes.c_double(0.0)
    rc = lib().vst_profile_read(int(kernel_class), ctypes.byref(n), ctypes.byref(ms))
    if rc < 0:
        raise ValueError("bad kernel class")
    return int(n.value), float(ms.value)


class VecchiaNLL(torch.autograd.Function):
    """NLL as a differentiable function of the 5 free native parameters.

    forward(theta5, fixed3, xy, t, y, nn, nn_cnt, m, precision, ws) where
    theta5 = (sigma1sq, c, a, gamma, nugget) is a float64 tensor (any device)
    and fixed3 = (alpha, delta, nu).  The gradient is computed by the
    library's adjoint kernel at forward time (the factor is recomputed, not
    stored) and scaled by grad_output in backward.
    """

    @staticmethod
    def forward(ctx, theta5, fixed3, xy, t, y, nn, nn_cnt, m, precision=MIXED, ws=None):
        th = [float(v) for v in theta5.detach().cpu().tolist()] + [float(v) for v in fixed3]
        nll, grad = vecchia_nll_grad(xy, t, th, m, nn, nn_cnt, y, precision=precision, ws=ws)
        ctx.save_for_backward(grad)
        ctx.theta_device = theta5.device
        return nll.reshape(()).to(theta5.device)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return (g * grad.to(ctx.theta_device),) + (None,) * 9
