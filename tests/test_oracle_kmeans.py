"""Pins for the oracle's K-means pieces against things other than itself.

* exact sums: ``math.fsum`` against exact rational arithmetic;
* d32: exact on small integers, and within the Higham bound gamma_{n+2} of
  the exact distance everywhere;
* assignment: against exact (Fraction) distances by brute force;
* Eq. (1) with k = 1 and the mean as centroid: the closed form
  sum ||x - mean||^2;
* Lloyd: sample objective non-increasing; agrees with scikit-learn's
  KMeans(algorithm="lloyd") iteration by iteration in pure64 mode;
* K-means++: candidate frequencies follow D^2 / sum D^2 (chi-square), the
  greedy choice is the brute-force least potential, weights are exact.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

from oracle import kmeans, rng


def _exact_dist(x, c):
    return sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(x, c))


def test_exact_sum_matches_fractions():
    g = np.random.default_rng(0)
    for trial in range(30):
        n = int(g.integers(1, 300))
        v = (g.standard_normal(n) * 10.0 ** g.integers(-30, 30, n)).astype(np.float32)
        if trial % 3 == 0:                                 # heavy cancellation
            v = np.concatenate([v, -v[: n // 2], np.float32([1e-30])])
        exact = sum(Fraction(float(x)) for x in v)
        assert kmeans.exact_sum(v) == float(exact)
    assert kmeans.exact_sum(np.float32([1e20, 1.0, -1e20])) == 1.0


def test_d32_exact_on_small_integers():
    g = np.random.default_rng(1)
    S = g.integers(-50, 50, (40, 7)).astype(np.float32)
    C = g.integers(-50, 50, (6, 7)).astype(np.float32)
    D = kmeans.d32_all(S, C)
    for i in range(40):
        for j in range(6):
            assert D[i, j] == float(_exact_dist(S[i], C[j]))


@pytest.mark.parametrize("n", [1, 2, 3, 16, 33])
def test_d32_within_higham_bound(n):
    g = np.random.default_rng(n)
    S = (g.standard_normal((30, n)) * 7 + 3).astype(np.float32)
    C = (g.standard_normal((5, n)) * 7).astype(np.float32)
    D = kmeans.d32_all(S, C)
    u = 2.0 ** -24
    gam = (n + 2) * u / (1 - (n + 2) * u)
    worst = 0.0
    for i in range(30):
        for j in range(5):
            ex = _exact_dist(S[i], C[j])
            err = abs(Fraction(float(D[i, j])) - ex)
            assert err <= Fraction(gam) * ex
            worst = max(worst, float(err / ex))
    assert worst > 0                                       # really computed in FP32


def test_assign_matches_exact_argmin():
    g = np.random.default_rng(2)
    S = (g.standard_normal((200, 3)) * 5).astype(np.float32)
    C = (g.standard_normal((7, 3)) * 5).astype(np.float32)
    lab, dist = kmeans.assign(S, C)
    for i in range(200):
        ex = [_exact_dist(S[i], c) for c in C]
        order = sorted(range(7), key=lambda j: ex[j])
        if (ex[order[1]] - ex[order[0]]) > Fraction(1, 10**4) * ex[order[0]]:
            assert lab[i] == order[0]


def test_assign_ties_go_to_lowest_index():
    S = np.float32([[0, 0], [1, 1], [5, 5]])
    C = np.float32([[1, 0], [0, 1], [1, 0], [5, 5]])       # duplicates and equidistant
    lab, _ = kmeans.assign(S, C)
    assert lab.tolist() == [0, 0, 3]


def test_objective_k1_closed_form():
    g = np.random.default_rng(3)
    X = (g.standard_normal((5000, 4)) * 3 + 1).astype(np.float32)
    mean = X.astype(np.float64).mean(axis=0)
    c = mean.astype(np.float32)[None, :]
    closed = float(((X.astype(np.float64) - c.astype(np.float64)) ** 2).sum())
    f = kmeans.objective(X, c)
    assert abs(f - closed) <= 1e-6 * closed
    assert kmeans.objective(X, c, "pure64") == pytest.approx(closed, rel=1e-12)


def test_objective_is_eq1_sum_of_minima():
    g = np.random.default_rng(4)
    X = (g.standard_normal((50, 2)) * 4).astype(np.float32)
    C = (g.standard_normal((3, 2)) * 4).astype(np.float32)
    brute = sum(min(_exact_dist(x, c) for c in C) for x in X)
    assert kmeans.objective(X, C) == pytest.approx(float(brute), rel=1e-6)


def _blobs(seed, m, n, k, spread=10.0):
    g = np.random.default_rng(seed)
    mu = g.uniform(-spread, spread, (k, n))
    lab = g.integers(0, k, m)
    return (mu[lab] + g.standard_normal((m, n))).astype(np.float32)


@pytest.mark.parametrize("mode", ["exact32", "pure64"])
def test_lloyd_objective_non_increasing(mode):
    X = _blobs(5, 3000, 5, 6)
    C0 = X[:6].copy()
    res = kmeans.lloyd(X, C0, max_iter=50, tol=-1.0, mode=mode)
    tr = np.array(res["trace"])
    slack = 0.0 if mode == "pure64" else 1e-6
    assert np.all(np.diff(tr) <= slack * tr[:-1] + 1e-300)
    assert res["iters"] == 50


def test_lloyd_matches_sklearn_pure64():
    sk = pytest.importorskip("sklearn.cluster")
    X = _blobs(6, 4000, 3, 5).astype(np.float64)
    C0 = X[[0, 10, 20, 30, 40]].copy()
    for t in (1, 2, 5, 12):
        km = sk.KMeans(n_clusters=5, init=C0, n_init=1, algorithm="lloyd", tol=0.0,
                       max_iter=t).fit(X)
        res = kmeans.lloyd(X, C0, max_iter=t, tol=-1.0, mode="pure64")
        if km.n_iter_ == t:
            np.testing.assert_allclose(res["C"], km.cluster_centers_, rtol=1e-12, atol=1e-12)
            assert res["f"] == pytest.approx(km.inertia_, rel=1e-10)


def test_lloyd_stop_rule_and_empty_clusters():
    X = np.float32([[0, 0], [0, 1], [10, 10], [10, 11]])
    C0 = np.float32([[0, 0.5], [10, 10.5], [100, 100]])    # third cluster never used
    res = kmeans.lloyd(X, C0, max_iter=300, tol=1e-4)
    assert res["iters"] == 1                                # converged immediately
    assert res["empty"].tolist() == [False, False, True]
    assert res["C"][2].tolist() == [100, 100]               # empty cluster keeps centroid
    assert res["f"] == 1.0


def test_quantised_weights_exact():
    D2 = np.float32([0.0, 1e-30, 0.75, 3.0, 2.9999998, 1.5])
    E = math.frexp(float(D2.max()))[1]
    w = kmeans.quantise(D2, E)
    for d, wi in zip(D2, w):
        assert wi == math.floor(Fraction(float(d)) * Fraction(2) ** (31 - E))
    assert w.max() < 2**31


def test_kmeanspp_first_candidate_distribution():
    # one live centroid at the origin; the first trial (l = 0) must pick
    # index i with probability w_i / sum(w).
    S = np.float32([[1, 0], [2, 0], [0, 3], [0.5, 0.5], [4, 0]])
    C = np.float32([[0, 0], [9, 9]])
    D2 = kmeans.d32_all(S, C[:1])[:, 0]
    E = math.frexp(float(D2.max()))[1]
    p = kmeans.quantise(D2, E).astype(np.float64)
    p /= p.sum()
    counts = np.zeros(5)
    for r in range(4000):
        key = rng.stream_key(r, rng.P_KPP, 0, 0, 0)
        _, picks = kmeans.kmeanspp_reseed(S, C, [False, True], key, n_trials=1)
        counts[picks[1]] += 1
    assert stats.chisquare(counts, p * counts.sum()).pvalue > 1e-4


def test_kmeanspp_greedy_picks_least_potential():
    g = np.random.default_rng(8)
    S = _blobs(8, 400, 2, 4)
    for r in range(20):
        key = rng.stream_key(r, rng.P_KPP, 1, 2, 3)
        C0 = np.zeros((4, 2), np.float32)
        C0[0] = S[g.integers(0, 400)]
        Cn, picks = kmeans.kmeanspp_reseed(S, C0, [False, True, True, True], key)
        # brute force the last centroid: recompute the three candidates
        D2 = np.min(kmeans.d32_all(S, Cn[:3]), axis=1)
        E = math.frexp(float(D2.max()))[1]
        w = kmeans.quantise(D2, E)
        pre = np.cumsum(w)
        cands = [int(np.argmax(pre > rng.draw_below(key, l, 3, int(pre[-1])))) for l in range(3)]
        pots = [int(kmeans.quantise(np.minimum(D2, kmeans.d32_all(S, S[c][None])[:, 0]), E).sum())
                for c in cands]
        assert picks[3] == cands[int(np.argmin(pots))]
        assert w[picks[3]] > 0


def test_kmeanspp_all_degenerate_first_is_uniform_draw():
    S = _blobs(9, 100, 3, 2)
    key = rng.stream_key(4, rng.P_KPP, 0, 0, 0)
    Cn, picks = kmeans.kmeanspp_reseed(S, np.zeros((2, 3), np.float32), [True, True], key)
    assert picks[0] == rng.draw_below(key, 0, 0, 100)
    assert np.array_equal(Cn[0], S[picks[0]])
    assert picks[1] != picks[0]
