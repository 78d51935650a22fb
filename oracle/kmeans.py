"""Space-time separated kMeans++ oracle (Algorithm 3).

TEST INFRASTRUCTURE (see oracle/__init__.py).  Plain numpy and Python
integers, one step at a time, for the small point sets Algorithm 3 works on
(the unique times and the unique locations).

Algorithm 3: m_s = round(sqrt(m n / |T|^2)) and m_t = round(sqrt(m |T|^2 / n))
(round = floor(x + 1/2); clamped to [1, |S|] and [1, |T|]) centres by kMeans++
on the unique locations S and the unique times T; the inducing points are the
Cartesian product S_bar x T_bar, point a m_t + b = (location a, time b).

kMeans++ (Arthur and Vassilvitskii, 2007) with the discrete choices made from
exact integers (a reading of the paper's kMeans++ step, chosen so that both sides
can agree bit for bit):
  * draws u_j = (mix(x0 + (j + 1) gamma) >> 11) 2^-53, SplitMix64 (Steele,
    Lea and Flood, 2014), x0 = seed (times) or seed ^ 0xD1B54A32D192ED03
    (locations);
  * first centre: point floor(u_0 N);
  * centre j: weights w_i = floor(D2_i * (2^32 / max D2)) as integers, the
    first point whose prefix sum exceeds min(floor(u_j * sum), sum - 1);
  * Lloyd step: nearest centre (ties to the smaller index); the new centre is
    the mean of the points quantised to q = rint((x - lo) * s), s = 2^32 /
    (hi - lo) (1 when hi == lo), summed as integers:
    centre = lo + (sum / count) / s; an empty cluster keeps its centre;
  * squared distances dx*dx + dy*dy (no fused multiply-add).

Pinned by (tests/test_oracle_kmeans.py): the published first outputs of
SplitMix64 from state 0; m_s m_t ~ m (the algorithm's stated property);
k = N picks every point once; well separated clusters give their means.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
LOC_STREAM = 0xD1B54A32D192ED03
M64 = (1 << 64) - 1
FIX = 4294967296.0  # 2^32


def mix(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def splitmix64(x0: int, j: int) -> int:
    """j-th output (0-based) of SplitMix64 started at state x0."""
    return mix((x0 + (j + 1) * GAMMA) & M64)


def uniform(x0: int, j: int) -> float:
    return (splitmix64(x0, j) >> 11) * 2.0 ** -53


def _d2(P, c):
    dx = P[:, 0] - c[0]
    dy = P[:, 1] - c[1]
    return dx * dx + dy * dy


def kmeanspp(P, k, x0, lloyd_iters):
    """Centres [k', 2] (k' = k unless all points are centres earlier)."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    N = P.shape[0]
    c0 = min(int(math.floor(uniform(x0, 0) * N)), N - 1)
    C = [P[c0].copy()]
    d2 = _d2(P, P[c0])
    for j in range(1, k):
        dmax = float(d2.max())
        if not dmax > 0.0:
            break
        s = FIX / dmax
        w = [int(math.floor(v)) for v in (d2 * s)]
        total = sum(w)
        target = min(int(math.floor(uniform(x0, j) * float(total))), total - 1)
        acc = 0
        idx = N - 1
        for i, wi in enumerate(w):
            acc += wi
            if acc > target:
                idx = i
                break
        C.append(P[idx].copy())
        d2 = np.minimum(d2, _d2(P, P[idx]))
    C = np.array(C)
    if lloyd_iters > 0:
        lo, hi = P.min(0), P.max(0)
        sq = np.array([FIX / (hi[d] - lo[d]) if hi[d] > lo[d] else 1.0 for d in range(2)])
        q = np.rint((P - lo) * sq)
        for _ in range(lloyd_iters):
            D = np.stack([_d2(P, c) for c in C], 1)
            a = np.argmin(D, 1)  # first minimum: the smaller centre index
            for j in range(C.shape[0]):
                sel = a == j
                cnt = int(sel.sum())
                if cnt == 0:
                    continue
                for d in range(2):
                    tot = sum(int(v) for v in q[sel, d])
                    C[j, d] = lo[d] + (float(tot) / float(cnt)) / sq[d]
    return C


def counts(n, n_times, m):
    """(m_s, m_t) before clamping."""
    ms = int(math.floor(math.sqrt(m * n / (n_times * n_times)) + 0.5))
    mt = int(math.floor(math.sqrt(m * n_times * n_times / n) + 0.5))
    return ms, mt


def sts_kmeanspp(xy, t, m, seed=0, lloyd_iters=10):
    """(xyk [k, 2], tk [k], (m_s, m_t))."""
    n = t.shape[0]
    T = np.unique(t)
    S = np.unique(np.ascontiguousarray(xy), axis=0)
    ms, mt = counts(n, T.shape[0], m)
    ms = min(max(ms, 1), S.shape[0])
    mt = min(max(mt, 1), T.shape[0])
    tc = kmeanspp(np.stack([T, np.zeros_like(T)], 1), mt, seed & M64, lloyd_iters)[:, 0]
    sc = kmeanspp(S, ms, (seed ^ LOC_STREAM) & M64, lloyd_iters)
    xyk = np.repeat(sc, tc.shape[0], axis=0)
    tk = np.tile(tc, sc.shape[0])
    return xyk, tk, (ms, mt)
