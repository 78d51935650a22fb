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


def test_counts_printed_formula():
    # Algorithm 3 (Sect. 4.4.2): m_s = round(sqrt(m n / |T|^2)) spatial and
    # m_t = round(sqrt(m |T|^2 / n)) temporal centres.  At n = 1,108,140,
    # |T| = 365, m = 1000: m n / |T|^2 = 8317.7 -> 91 and m |T|^2 / n = 120.2
    # -> 11; swapping the two formulas gives (11, 91) and fails.
    assert okm.counts(1_108_140, 365, 1000) == (91, 11)
    # more data per time point than time points: more spatial centres
    assert okm.counts(2_000, 10, 100) == (45, 2)
    # round = floor(x + 1/2): sqrt(m n / |T|^2) = 2.5 exactly rounds up
    assert okm.counts(625, 10, 1) == (3, 0)


def test_kmeanspp_second_centre_follows_d2():
    # kMeans++ seeding (Arthur and Vassilvitskii 2007): after the first centre,
    # the next one is drawn with probability proportional to the squared
    # distance D^2 to the nearest chosen centre.  Points on a line at 0, 1, 3:
    # with the first centre at 0, D^2 = (0, 1, 9), so the point at 1 is chosen
    # with probability 0.1 (D weighting would give 0.25, uniform 0.5).
    P = np.array([[0.0, 0.0], [1.0, 0.0], [3.0, 0.0]])
    hits, total = 0, 0
    for seed in range(3000):
        C = okm.kmeanspp(P, 2, seed, 0)
        if C[0, 0] != 0.0:
            continue
        total += 1
        assert C[1, 0] in (1.0, 3.0)
        hits += C[1, 0] == 1.0
    assert total > 700
    frac = hits / total
    # binomial standard deviation at p = 0.1 and ~1000 draws is ~0.01
    assert abs(frac - 0.1) < 0.04, frac


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
