"""Vecchia prediction oracle (the predictive distribution of Sect. 3.1 under
the Vecchia approximation, Sect. 4.1, with the correlation neighbours of
Sect. 4.4.1).

TEST INFRASTRUCTURE (see oracle/__init__.py).  Plain numpy/scipy, FP64, for
small inputs: a dense correlation matrix between prediction and training
points, and one dense local solve per prediction point.

Reading of Sect. 3.1 under the Vecchia approximation: every prediction point conditions on the
min(m, n) training points with the largest correlation C(p, j) / sigma1^2
(latent covariance, no nugget; ties to the smaller training index; sorted by
decreasing correlation); prediction points do not condition on one another.
Then, with Sigma~ = Sigma + nugget I on the local block,
    mean_p = Sigma~_{p,N} Sigma~_N^{-1} y_N,
    var_p  = Sigma~_pp - Sigma~_{p,N} Sigma~_N^{-1} Sigma~_{N,p}   (response),
and the latent variance is var_p - nugget.

Pinned by (tests/test_oracle_predict.py): with m = n every training point is
a neighbour and the result is the exact kriging predictor of Sect. 3.1
(computed from one Cholesky factor of the full training covariance); variances
lie in (0, sigma1^2 + nugget]; a prediction point far from every training
point returns the prior (mean 0, variance sigma1^2 + nugget).
"""
from __future__ import annotations

import numpy as np

from . import cov_matrix


def neighbours(xy, t, xyp, tp, theta, m):
    """nn [np, m] int32 (-1 padded), cnt [np]: training points by decreasing
    correlation, ties to the smaller index."""
    n, npred = t.shape[0], tp.shape[0]
    c = min(m, n)
    nn = np.full((npred, m), -1, dtype=np.int32)
    cnt = np.full(npred, c, dtype=np.int32)
    if c == 0:
        return nn, cnt
    R = cov_matrix(xyp, tp, xy, t, theta) / theta[0]
    j = np.arange(n)
    for p in range(npred):
        order = np.lexsort((j, -R[p]))
        nn[p, :c] = order[:c]
    return nn, cnt


def predict(xy, t, y, xyp, tp, theta, m, latent=False):
    """(mean [np], var [np], nn [np, m])."""
    nn, cnt = neighbours(xy, t, xyp, tp, theta, m)
    npred = tp.shape[0]
    mean = np.zeros(npred)
    var = np.zeros(npred)
    prior = theta[0] + theta[4]
    for p in range(npred):
        N = nn[p, :cnt[p]].astype(np.int64)
        if N.size == 0:
            mean[p], var[p] = 0.0, prior
        else:
            KN = cov_matrix(xy[N], t[N], xy[N], t[N], theta) + theta[4] * np.eye(N.size)
            k = cov_matrix(xy[N], t[N], xyp[p:p + 1], tp[p:p + 1], theta)[:, 0]
            a = np.linalg.solve(KN, k)
            mean[p] = a @ y[N]
            var[p] = prior - a @ k
        if latent:
            var[p] -= theta[4]
    return mean, var, nn
