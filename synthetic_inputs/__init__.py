"""Seeded synthetic inputs shaped like the paper's station data.

This module is shared by the CPU oracle's tests and the CUDA path's tests and
benchmark.  It holds no covariance, likelihood or Vecchia arithmetic: it draws
station coordinates, observation days, missing-value masks, orderings,
standard-normal variates and inducing-point locations (plain kMeans++ on
scaled Euclidean coordinates), and returns them as numpy arrays.  Responses
that need the covariance (exact or Vecchia sampling) are produced by whichever
side is under test from the variates drawn here.

Workloads (all seeded; every number below is a parameter of the recipe):

* ``tiny_uniform``  -- 200 stations uniform on [0,1]^2 x 10 integer days
  (n = 2,000), fully random ordering.
* ``box_uniform``   -- 1,000 stations uniform in a 58 x 24 degree lon/lat box,
  scaled by the box width, x 100 days (n = 100,000), time-stratified order.
* ``continental``   -- 3,300 stations from a 40-component Gaussian mixture
  (sigma = 2 degrees) in the same box x 365 days, 8% of station-days dropped
  at random (n ~ 1.108M), time-stratified order.
* ``batched``       -- 64 independent datasets with n_d log-uniform in
  [5e3, 5e4], 50 days each, per-dataset covariance ranges.

The paper's own data (NOAA GHCNd station records, the 2nd spatial statistics
competition sets) are not available; these stand in for them with the same
shapes: a few thousand irregular stations observed daily (Sect. 2, Sect. 6)
and up to ~1.2M space-time points.
"""
from __future__ import annotations

import dataclasses
import numpy as np

# lon/lat box of the contiguous US used for the station layouts (degrees)
LON0, LON1 = -125.0, -67.0
LAT0, LAT1 = 25.0, 49.0
BOX_W = LON1 - LON0  # 58 degrees: coordinates are divided by this width


@dataclasses.dataclass
class RangeTheta:
    """Covariance parameters in 'effective range' form.

    sigma2: marginal variance sigma_1^2 of the latent process.
    range_s: spatial distance at which the zero-lag correlation is 0.05.
    range_t: time lag at which the zero-distance correlation is 0.05.
    gamma: non-separability (interaction) parameter in [0, 1].
    nugget: variance sigma^2 of the independent noise.
    alpha, delta, nu: fixed shape parameters.
    """
    sigma2: float = 1.0
    range_s: float = 0.1
    range_t: float = 3.0
    gamma: float = 0.5
    nugget: float = 0.05
    alpha: float = 0.4
    delta: float = 0.2
    nu: float = 1.5

    def astuple(self):
        return (self.sigma2, self.range_s, self.range_t, self.gamma, self.nugget,
                self.alpha, self.delta, self.nu)


@dataclasses.dataclass
class Workload:
    """Points already permuted into Vecchia order."""
    name: str
    xy: np.ndarray        # float64 [n, 2]
    t: np.ndarray         # float64 [n]
    z: np.ndarray         # float64 [n] standard-normal variates for response simulation
    theta: RangeTheta
    m: int
    order: np.ndarray     # int64 [n]: row r of xy/t is original point order[r]
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.t.shape[0])


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


def stations_uniform(n_st: int, seed: int) -> np.ndarray:
    return _rng(seed).random((n_st, 2))


def stations_box_uniform(n_st: int, seed: int) -> np.ndarray:
    r = _rng(seed)
    lon = r.uniform(LON0, LON1, n_st)
    lat = r.uniform(LAT0, LAT1, n_st)
    return np.stack([(lon - LON0) / BOX_W, (lat - LAT0) / BOX_W], axis=1)


def stations_clustered(n_st: int, seed: int, n_clusters: int = 40, sigma_deg: float = 2.0) -> np.ndarray:
    """Mixture of isotropic Gaussians (centres uniform in the box); draws that
    fall outside the box are redrawn."""
    r = _rng(seed)
    clon = r.uniform(LON0, LON1, n_clusters)
    clat = r.uniform(LAT0, LAT1, n_clusters)
    out = np.empty((n_st, 2))
    for s in range(n_st):
        k = r.integers(n_clusters)
        while True:
            lon = clon[k] + sigma_deg * r.standard_normal()
            lat = clat[k] + sigma_deg * r.standard_normal()
            if LON0 <= lon <= LON1 and LAT0 <= lat <= LAT1:
                break
        out[s] = ((lon - LON0) / BOX_W, (lat - LAT0) / BOX_W)
    return out


def station_days(stations: np.ndarray, n_days: int):
    """All (station, day) pairs, day-major: returns xy [S*T, 2], t [S*T]."""
    S = stations.shape[0]
    xy = np.tile(stations, (n_days, 1))
    t = np.repeat(np.arange(n_days, dtype=np.float64), S)
    return xy, t


def drop_random(n: int, frac: float, seed: int) -> np.ndarray:
    """Boolean keep-mask with round(frac*n) entries dropped uniformly at random."""
    r = _rng(seed)
    keep = np.ones(n, dtype=bool)
    keep[r.choice(n, size=int(round(frac * n)), replace=False)] = False
    return keep


def random_order(n: int, seed: int) -> np.ndarray:
    return _rng(seed).permutation(n).astype(np.int64)


def time_stratified_order(t: np.ndarray, seed: int) -> np.ndarray:
    """Sort by time; within each time point, a random permutation (Sect. 4.4.1)."""
    r = _rng(seed)
    key = r.random(t.shape[0])
    return np.lexsort((key, t)).astype(np.int64)


def standard_normal(n: int, seed: int) -> np.ndarray:
    return _rng(seed).standard_normal(n)


def _finish(name, xy, t, order, theta, m, z_seed, meta=None) -> Workload:
    xy = np.ascontiguousarray(xy[order])
    t = np.ascontiguousarray(t[order])
    return Workload(name=name, xy=xy, t=t, z=standard_normal(t.shape[0], z_seed),
                    theta=theta, m=m, order=order, meta=meta or {})


def tiny_uniform(seed: int = 0, m: int = 10) -> Workload:
    """200 stations on [0,1]^2 x days 0..9 (n=2,000), fully random order."""
    st = stations_uniform(200, seed)
    xy, t = station_days(st, 10)
    order = random_order(t.shape[0], seed)
    th = RangeTheta(sigma2=1.0, range_s=0.1, range_t=3.0, gamma=0.5, nugget=0.05)
    return _finish("tiny_uniform_n2000", xy, t, order, th, m, seed + 1000)


def box_uniform(seed: int = 2, m: int = 20, n_st: int = 1000, n_days: int = 100) -> Workload:
    """1,000 stations uniform in the lon/lat box x 100 days, time-stratified."""
    st = stations_box_uniform(n_st, seed)
    xy, t = station_days(st, n_days)
    order = time_stratified_order(t, seed)
    th = RangeTheta(sigma2=1.0, range_s=0.08, range_t=3.0, gamma=0.5, nugget=0.05)
    return _finish(f"box_uniform_n{t.shape[0]}", xy, t, order, th, m, seed + 1000)


def continental(seed: int = 3, m: int = 30, n_st: int = 3300, n_days: int = 365,
                drop: float = 0.08) -> Workload:
    """3,300 clustered stations x 365 days with 8% of station-days missing."""
    st = stations_clustered(n_st, seed)
    xy, t = station_days(st, n_days)
    keep = drop_random(t.shape[0], drop, seed + 7)
    xy, t = xy[keep], t[keep]
    order = time_stratified_order(t, seed)
    th = RangeTheta(sigma2=1.0, range_s=0.08, range_t=3.0, gamma=0.5, nugget=0.05)
    return _finish(f"continental_n{t.shape[0]}", xy, t, order, th, m, seed + 1000)


def batched(seed: int = 5, n_sets: int = 64, m: int = 20, n_days: int = 50,
            n_lo: float = 5e3, n_hi: float = 5e4):
    """64 independent datasets (n_d log-uniform in [5e3, 5e4]); each has its own
    ranges drawn uniformly: range_s in [.05,.3], range_t in [1,10], gamma in
    [.1,.9], nugget in [.01,.2]; sigma_1^2 = 1."""
    r = _rng(seed)
    sets = []
    for d in range(n_sets):
        n_d = int(round(np.exp(r.uniform(np.log(n_lo), np.log(n_hi)))))
        n_st = int(np.ceil(n_d / n_days))
        st = r.random((n_st, 2))
        xy, t = station_days(st, n_days)
        extra = t.shape[0] - n_d
        keep = np.ones(t.shape[0], dtype=bool)
        if extra > 0:
            keep[r.choice(t.shape[0], size=extra, replace=False)] = False
        xy, t = xy[keep], t[keep]
        th = RangeTheta(sigma2=1.0, range_s=r.uniform(0.05, 0.3), range_t=r.uniform(1, 10),
                        gamma=r.uniform(0.1, 0.9), nugget=r.uniform(0.01, 0.2))
        order = time_stratified_order(t, seed * 1000 + d)
        sets.append(_finish(f"batched_{d}", xy, t, order, th, m, seed * 1000 + 500 + d))
    return sets


def kmeanspp(X: np.ndarray, k: int, seed: int, lloyd_iters: int = 100) -> np.ndarray:
    """Plain kMeans++ seeding (D^2 sampling) followed by Lloyd iterations until
    the assignment stops changing or ``lloyd_iters`` is reached.  Euclidean
    distances on the given (already scaled) coordinates."""
    r = _rng(seed)
    n = X.shape[0]
    C = np.empty((k, X.shape[1]))
    C[0] = X[r.integers(n)]
    d2 = ((X - C[0]) ** 2).sum(1)
    for j in range(1, k):
        p = d2 / d2.sum()
        C[j] = X[r.choice(n, p=p)]
        d2 = np.minimum(d2, ((X - C[j]) ** 2).sum(1))
    assign = None
    for _ in range(lloyd_iters):
        # nearest centre in chunks (n*k distances)
        new = np.empty(n, dtype=np.int64)
        cn = (C ** 2).sum(1)
        for s in range(0, n, 65536):
            Xs = X[s:s + 65536]
            dd = (Xs ** 2).sum(1)[:, None] - 2 * Xs @ C.T + cn[None, :]
            new[s:s + 65536] = dd.argmin(1)
        if assign is not None and np.array_equal(new, assign):
            break
        assign = new
        for j in range(k):
            sel = assign == j
            if sel.any():
                C[j] = X[sel].mean(0)
    return C


def inducing_points(w: Workload, k: int, seed: int = 11, lloyd_iters: int = 20):
    """Space-time kMeans++ (+ Lloyd) on (x/range_s, y/range_s, t/range_t);
    returns (xy [k,2], t [k]) in the original units."""
    th = w.theta
    X = np.concatenate([w.xy / th.range_s, (w.t / th.range_t)[:, None]], axis=1)
    C = kmeanspp(X, k, seed, lloyd_iters)
    return np.ascontiguousarray(C[:, :2] * th.range_s), np.ascontiguousarray(C[:, 2] * th.range_t)
