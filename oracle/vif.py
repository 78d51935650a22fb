"""VIF oracle: the Vecchia-inducing-point full-scale approximation (Sect. 4.3).

TEST INFRASTRUCTURE (see oracle/__init__.py).  Plain numpy/scipy, FP64, for
small n (dense k x k algebra, per-row loops).  Library primitives (Cholesky,
triangular solve) are used as steps; everything else is written out.

Model (the reading of Sect. 4.3 taken here): the latent process is b = b_l + b_s
with the predictive-process part Cov(b_l) = Sigma_nk Sigma_kk^{-1} Sigma_kn
(k inducing points) and the residual Cov(b_s) = Sigma - Sigma_nk Sigma_kk^{-1}
Sigma_kn.  The residual plus the nugget, R~ = Cov(b_s) + sigma^2 I, is
Vecchia-approximated with the residual coefficients A_i, D_i of Sect. 4.3
(nugget on the diagonal), so the response covariance is

    Sigma~_VIF = U U^T + B^{-1} D B^{-T},   U = Sigma_nk L_kk^{-T},  L_kk L_kk^T = Sigma_kk.

Neighbours are chosen by the residual correlation |R_ij| / sqrt(R_ii R_jj)
(the d_c metric of Sect. 4.4.1 applied to Cov(b_s), no nugget).  The NLL is
evaluated with the Sherman-Woodbury-Morrison identity (the complexity remark
at the end of Sect. 4.3):

    W = D^{-1/2} B U,  e = D^{-1/2} B y,  M = I_k + W^T W,
    log det Sigma~_VIF = sum_i log D_i + log det M,
    y^T Sigma~_VIF^{-1} y = e^T e - (W^T e)^T M^{-1} (W^T e).

Pinned by (tests/test_oracle_vif.py): m = n-1 gives the exact GP likelihood
for any k; k = 0 gives plain Vecchia; m = 0 gives the dense FITC likelihood
(Sect. 4.2); the Woodbury value equals the dense Sigma~_VIF likelihood.

The gradient (nll_grad) is the derivative of that NLL with the neighbour sets
and inducing points held fixed, taken in forward mode on dense matrices: one
derivative of every intermediate (Sigma_kk, L_kk, U, R~, A_i, D_i, B^{-1},
Sigma~_VIF) per parameter, then 1/2 tr(Sigma~^{-1} dSigma~) - 1/2 alpha^T
dSigma~ alpha.  Pinned by (tests/test_oracle_vif.py): central differences of
nll; k = 0 gives the plain Vecchia gradient; m = n-1 gives the exact GP
gradient for any k.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import cov_grad, cov_matrix


def lowrank(xy, t, xyk, tk, theta):
    """U = Sigma_nk L_kk^{-T} (n x k), residual variances r_i = Sigma_ii - ||U_i||^2."""
    n, k = t.shape[0], (tk.shape[0] if tk is not None else 0)
    if k == 0:
        return np.zeros((n, 0)), np.full(n, theta[0])
    Skk = cov_matrix(xyk, tk, xyk, tk, theta)
    Snk = cov_matrix(xy, t, xyk, tk, theta)
    L = np.linalg.cholesky(Skk)
    U = sla.solve_triangular(L, Snk.T, lower=True).T
    r = theta[0] - (U * U).sum(1)
    return U, r


def lowrank_rows(xy, t, xyk, tk, theta, chunk=32768, threads=None):
    """The same U and r as lowrank() for large n: the rows of Sigma_nk are
    formed and solved in independent chunks of points (rows of U do not
    depend on one another), the chunks' covariance matrices in parallel
    threads (the C++ covariance releases the interpreter)."""
    from concurrent.futures import ThreadPoolExecutor
    from . import default_threads
    n, k = t.shape[0], tk.shape[0]
    Skk = cov_matrix(xyk, tk, xyk, tk, theta)
    L = np.linalg.cholesky(Skk)
    U = np.empty((n, k))
    starts = list(range(0, n, chunk))

    def one(s):
        e = min(n, s + chunk)
        Snk = cov_matrix(xy[s:e], t[s:e], xyk, tk, theta)
        U[s:e] = sla.solve_triangular(L, Snk.T, lower=True).T

    with ThreadPoolExecutor(threads or default_threads()) as ex:
        list(ex.map(one, starts))
    r = theta[0] - (U * U).sum(1)
    return U, r


def knn_rows(xy, t, theta, U, r, m, rows):
    """knn() for the listed rows only (brute force over all their
    predecessors): (nn [len(rows), m], cnt, rho_m, rho_m1)."""
    rows = np.asarray(rows, dtype=np.int64)
    nn = np.full((rows.shape[0], m), -1, dtype=np.int32)
    cnt = np.zeros(rows.shape[0], dtype=np.int32)
    rm = np.full(rows.shape[0], np.nan)
    rm1 = np.full(rows.shape[0], np.nan)
    tiny = 1e-12 * theta[0]
    for q, i in enumerate(rows):
        if i == 0:
            continue
        j = np.arange(i)
        R = cov_matrix(xy[i:i + 1], t[i:i + 1], xy[:i], t[:i], theta)[0] - U[:i] @ U[i]
        ok = (r[j] > tiny) & (r[i] > tiny)
        rho = np.where(ok, np.abs(R) / np.sqrt(np.where(ok, r[i] * r[j], 1.0)), 0.0)
        order = np.lexsort((j, -rho))
        c = min(int(i), m)
        nn[q, :c] = j[order[:c]]
        cnt[q] = c
        if c == m and m > 0:
            rm[q] = rho[order[m - 1]]
        if i > m:
            rm1[q] = rho[order[m]]
    return nn, cnt, rm, rm1


def residual_block(xy, t, theta, U, rows, cols):
    """Latent residual covariance R[rows, cols] = Sigma - U U^T (no nugget)."""
    C = cov_matrix(xy[rows], t[rows], xy[cols], t[cols], theta)
    return C - U[rows] @ U[cols].T


def knn(xy, t, theta, U, r, m):
    """Brute-force residual-correlation neighbours: for each i, the min(i, m)
    predecessors with the largest |R_ij| / sqrt(R_ii R_jj); ties -> smaller
    index; sorted by decreasing |rho|.  A point whose residual variance is at
    most 1e-12 sigma1^2 (an inducing point on top of it) has no defined
    residual correlation; it is taken as 0 (a reading: the paper is silent).
    Returns nn, cnt, rho_m, rho_m1."""
    n = t.shape[0]
    nn = np.full((n, m), -1, dtype=np.int32)
    cnt = np.zeros(n, dtype=np.int32)
    rm = np.full(n, np.nan)
    rm1 = np.full(n, np.nan)
    for i in range(1, n):
        j = np.arange(i)
        R = residual_block(xy, t, theta, U, np.array([i]), j)[0]
        tiny = 1e-12 * theta[0]
        ok = (r[j] > tiny) & (r[i] > tiny)
        rho = np.where(ok, np.abs(R) / np.sqrt(np.where(ok, r[i] * r[j], 1.0)), 0.0)
        order = np.lexsort((j, -rho))
        c = min(i, m)
        nn[i, :c] = j[order[:c]]
        cnt[i] = c
        if c == m and m > 0:
            rm[i] = rho[order[m - 1]]
        if i > m:
            rm1[i] = rho[order[m]]
    return nn, cnt, rm, rm1


def factor(xy, t, theta, U, m, nn, cnt):
    """Residual Vecchia factor of R~ = R + sigma^2 I (Sect. 4.3): A_i, D_i."""
    n = t.shape[0]
    A = np.zeros((n, m))
    D = np.zeros(n)
    for i in range(n):
        N = nn[i, :cnt[i]].astype(np.int64)
        Rii = residual_block(xy, t, theta, U, np.array([i]), np.array([i]))[0, 0] + theta[4]
        if N.size == 0:
            D[i] = Rii
            continue
        RN = residual_block(xy, t, theta, U, N, N) + theta[4] * np.eye(N.size)
        k = residual_block(xy, t, theta, U, N, np.array([i]))[:, 0]
        a = np.linalg.solve(RN, k)
        A[i, :N.size] = a
        D[i] = Rii - a @ k
    return A, D


def nll(xy, t, theta, U, m, nn, cnt, y, A=None, D=None):
    """VIF negative log-likelihood by the Woodbury identity (see module doc)."""
    n, k = t.shape[0], U.shape[1]
    if A is None:
        A, D = factor(xy, t, theta, U, m, nn, cnt)
    By = y.copy()
    BU = U.copy()
    for i in range(n):
        N = nn[i, :cnt[i]].astype(np.int64)
        if N.size:
            By[i] -= A[i, :N.size] @ y[N]
            BU[i] -= A[i, :N.size] @ U[N]
    s = 1.0 / np.sqrt(D)
    e = By * s
    W = BU * s[:, None]
    M = np.eye(k) + W.T @ W
    Lm = np.linalg.cholesky(M) if k else np.zeros((0, 0))
    z = sla.solve_triangular(Lm, W.T @ e, lower=True) if k else np.zeros(0)
    logdet = np.log(D).sum() + 2.0 * np.log(np.diag(Lm)).sum()
    quad = e @ e - z @ z
    return 0.5 * n * np.log(2 * np.pi) + 0.5 * logdet + 0.5 * quad


def dense_sigma(xy, t, theta, U, m, nn, cnt, A=None, D=None):
    """Sigma~_VIF = U U^T + B^{-1} D B^{-T} formed densely (small n)."""
    n = t.shape[0]
    if A is None:
        A, D = factor(xy, t, theta, U, m, nn, cnt)
    B = np.eye(n)
    for i in range(n):
        B[i, nn[i, :cnt[i]]] = -A[i, :cnt[i]]
    Binv = sla.solve_triangular(B, np.eye(n), lower=True)
    return U @ U.T + Binv @ np.diag(D) @ Binv.T


def _dcov(xy1, t1, xy2, t2, theta):
    """d Sigma(x1, x2) / d(sigma1^2, c, a, gamma) as [4, n1, n2] (no nugget)."""
    n1, n2 = t1.shape[0], t2.shape[0]
    out = np.zeros((4, n1, n2))
    for i in range(n1):
        for j in range(n2):
            h = float(np.hypot(xy1[i, 0] - xy2[j, 0], xy1[i, 1] - xy2[j, 1]))
            out[:, i, j] = cov_grad(theta, h, float(t1[i] - t2[j]))
    return out


def nll_grad(xy, t, theta, xyk, tk, m, nn, cnt, y):
    """VIF NLL and its gradient w.r.t. (sigma1^2, c, a, gamma, nugget), the
    neighbour sets and inducing points held fixed (forward mode, dense; small n)."""
    xy, t, y = np.asarray(xy, float), np.asarray(t, float), np.asarray(y, float)
    n = t.shape[0]
    k = 0 if tk is None else tk.shape[0]
    theta = np.asarray(theta, float)
    # low rank and its derivatives: U L^T = Sigma_nk, dL = L Phi(L^{-1} dSigma_kk L^{-T})
    if k:
        Skk = cov_matrix(xyk, tk, xyk, tk, theta)
        Snk = cov_matrix(xy, t, xyk, tk, theta)
        L = np.linalg.cholesky(Skk)
        Linv = sla.solve_triangular(L, np.eye(k), lower=True)
        U = Snk @ Linv.T
        dSkk = _dcov(xyk, tk, xyk, tk, theta)
        dSnk = _dcov(xy, t, xyk, tk, theta)
    else:
        U = np.zeros((n, 0))
    dU = np.zeros((5, n, k))
    for j in range(4):
        if not k:
            break
        Z = Linv @ dSkk[j] @ Linv.T
        Phi = np.tril(Z) - 0.5 * np.diag(np.diag(Z))
        dL = L @ Phi
        dU[j] = (dSnk[j] - U @ dL.T) @ Linv.T
    # residual plus nugget and its derivatives
    C = cov_matrix(xy, t, xy, t, theta)
    dC = _dcov(xy, t, xy, t, theta)
    Rt = C - U @ U.T + theta[4] * np.eye(n)
    dRt = np.zeros((5, n, n))
    for j in range(5):
        if j < 4:
            dRt[j] = dC[j] - dU[j] @ U.T - U @ dU[j].T
        else:
            dRt[j] = np.eye(n)
    # residual Vecchia factor and its derivatives, row by row
    A = np.zeros((n, m))
    D = np.zeros(n)
    dA = np.zeros((5, n, m))
    dD = np.zeros((5, n))
    for i in range(n):
        N = nn[i, :cnt[i]].astype(np.int64)
        c = N.size
        if c == 0:
            D[i] = Rt[i, i]
            dD[:, i] = dRt[:, i, i]
            continue
        KN = Rt[np.ix_(N, N)]
        kv = Rt[N, i]
        a = np.linalg.solve(KN, kv)
        A[i, :c] = a
        D[i] = Rt[i, i] - kv @ a
        for j in range(5):
            dKN = dRt[j][np.ix_(N, N)]
            dk = dRt[j][N, i]
            dA[j, i, :c] = np.linalg.solve(KN, dk - dKN @ a)
            dD[j, i] = dRt[j][i, i] - 2.0 * dk @ a + a @ dKN @ a
    B = np.eye(n)
    for i in range(n):
        B[i, nn[i, :cnt[i]]] = -A[i, :cnt[i]]
    Binv = sla.solve_triangular(B, np.eye(n), lower=True)
    S = Binv @ np.diag(D) @ Binv.T
    Sig = U @ U.T + S
    Lf = np.linalg.cholesky(Sig)
    alpha = sla.cho_solve((Lf, True), y)
    Sinv = sla.cho_solve((Lf, True), np.eye(n))
    value = 0.5 * n * np.log(2 * np.pi) + np.log(np.diag(Lf)).sum() + 0.5 * y @ alpha
    grad = np.zeros(5)
    for j in range(5):
        dAm = np.zeros((n, n))
        for i in range(n):
            dAm[i, nn[i, :cnt[i]]] = dA[j, i, :cnt[i]]
        dBinv = Binv @ dAm @ Binv  # B = I - A
        dS = dBinv @ np.diag(D) @ Binv.T + Binv @ np.diag(dD[j]) @ Binv.T + Binv @ np.diag(D) @ dBinv.T
        dSig = dU[j] @ U.T + U @ dU[j].T + dS
        grad[j] = 0.5 * np.sum(Sinv * dSig) - 0.5 * alpha @ dSig @ alpha
    return value, grad
