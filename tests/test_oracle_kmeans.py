"""Pins of the space-time separated kMeans++ oracle (oracle/kmeans.py)."""
import numpy as np

import oracle.kmeans as okm
import synthetic_inputs as si


def test_splitmix64_published_outputs():
    # the first two outputs of SplitMix64 (Steele, Lea and Flood 2014) from
    # state 0, as printed by its reference implementation
    assert okm.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert okm.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert 0.0 <= okm.uniform(0, 0) < 1.0


def test_counts_multiply_to_m():
    # Algorithm 3: m_hat = m_s m_t ~ m
    for n, nt, m in [(1000, 10, 100), (1_108_140, 365, 1000), (50_000, 50, 250), (5_000, 100, 60)]:
        ms, mt = okm.counts(n, nt, m)
        assert abs(ms * mt - m) <= 0.3 * m


def test_every_point_a_centre_when_k_equals_n():
    P = np.random.default_rng(4).random((40, 2))
    C = okm.kmeanspp(P, 40, 123, 0)
    assert C.shape == (40, 2)
    assert {tuple(c) for c in C} == {tuple(p) for p in P}


def test_separated_clusters_give_their_means():
    rng = np.random.default_rng(5)
    centres = np.array([[0, 0], [10, 0], [0, 10], [10, 10]], dtype=float)
    lab = rng.integers(0, 4, 400)
    P = centres[lab] + 1e-3 * rng.standard_normal((400, 2))
    C = okm.kmeanspp(P, 4, 77, 5)
    means = np.array([P[lab == j].mean(0) for j in range(4)])
    # one centre per cluster, each at its cluster's mean (to the 2^-32 quantisation)
    order = [int(np.argmin(((C - mu) ** 2).sum(1))) for mu in means]
    assert sorted(order) == [0, 1, 2, 3]
    np.testing.assert_allclose(C[order], means, atol=1e-8)


def test_lloyd_does_not_increase_the_within_cluster_sum_of_squares():
    P = np.random.default_rng(6).random((300, 2))

    def wss(C):
        return (np.stack([((P - c) ** 2).sum(1) for c in C], 1).min(1)).sum()

    last = wss(okm.kmeanspp(P, 12, 9, 0))
    for it in (1, 2, 5, 10):
        cur = wss(okm.kmeanspp(P, 12, 9, it))
        assert cur <= last * (1 + 1e-9)
        last = cur


def test_product_layout():
    w = si.tiny_uniform()
    xyk, tk, (ms, mt) = okm.sts_kmeanspp(w.xy, w.t, 40, seed=3, lloyd_iters=2)
    assert xyk.shape == (ms * mt, 2) and tk.shape == (ms * mt,)
    assert len(np.unique(tk)) == mt and len(np.unique(xyk, axis=0)) == ms
    assert np.all(xyk[1] == xyk[0]) if mt > 1 else True
