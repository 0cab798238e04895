"""Pins for the oracle's Algorithm 1 (competitive sample size Big-means).

* brute-force optimal partitions (all k^m labelings) for m <= 10, k <= 3:
  Big-means never beats the optimum and reaches it on separated data;
* the closed-form 1-D two-cluster optimum (best contiguous split of the
  sorted points);
* the incumbent rule of Sec. 4.1: within a round f_hat_w never increases,
  and the tracked full-data incumbent never increases;
* s_opt is the rounded mean of the improving sizes L (Sec. 4.2) and every
  entry of L is a size that was drawn;
* W = 1, p = 1, T = 1, s = m reduces to K-means++ followed by Lloyd on X.
"""
import itertools

import numpy as np
import pytest

from oracle import bigmeans, kmeans, rng

BUDGET = dict(rounds=2, max_lloyd=300, tol=1e-4, kpp_candidates=3)


def _brute_opt(X, k):
    X = X.astype(np.float64)
    m = X.shape[0]
    best = np.inf
    for lab in itertools.product(range(k), repeat=m):
        lab = np.array(lab)
        f = 0.0
        for j in range(k):
            P = X[lab == j]
            if len(P):
                f += float(((P - P.mean(axis=0)) ** 2).sum())
        best = min(best, f)
    return best


@pytest.mark.parametrize("seed,m,k,sep", [(0, 8, 2, 0.0), (1, 9, 3, 0.0), (2, 10, 3, 30.0),
                                          (3, 10, 2, 30.0), (4, 7, 3, 1.0)])
def test_never_below_brute_force_optimum(seed, m, k, sep):
    g = np.random.default_rng(seed)
    centers = g.uniform(-1, 1, (k, 2)) * sep
    X = (centers[g.integers(0, k, m)] + g.standard_normal((m, 2))).astype(np.float32)
    f_opt = _brute_opt(X, k)
    res = bigmeans.bigmeans(X, k, dict(s_min=max(k, m // 2), s_max=m, workers=3, passes=4),
                            BUDGET, seed=seed)
    assert res["f_full"] >= f_opt * (1 - 1e-6)


def test_reaches_optimum_on_separated_data():
    g = np.random.default_rng(10)
    centers = np.array([[-40.0, 0.0], [0.0, 40.0], [40.0, 0.0]])
    X = (centers[np.arange(9) % 3] + 0.5 * g.standard_normal((9, 2))).astype(np.float32)
    f_opt = _brute_opt(X, 3)
    res = bigmeans.bigmeans(X, 3, dict(s_min=9, s_max=9, workers=2, passes=3), BUDGET, seed=1)
    assert res["f_full"] == pytest.approx(f_opt, rel=1e-6)


def test_one_dimensional_two_cluster_closed_form():
    g = np.random.default_rng(11)
    x = np.concatenate([g.normal(-6, 1, 300), g.normal(5, 1.5, 500)]).astype(np.float32)
    xs = np.sort(x.astype(np.float64))
    c1 = np.cumsum(xs)
    c2 = np.cumsum(xs ** 2)
    m = len(xs)
    best = np.inf
    for i in range(1, m):                  # left = xs[:i], right = xs[i:]
        sl, ql = c1[i - 1], c2[i - 1]
        sr, qr = c1[-1] - sl, c2[-1] - ql
        best = min(best, (ql - sl * sl / i) + (qr - sr * sr / (m - i)))
    # with s = m every sample is all of X and Lloyd runs to its fixed point
    res = bigmeans.bigmeans(x[:, None], 2, dict(s_min=m, s_max=m, workers=3, passes=2),
                            dict(BUDGET, tol=0.0), seed=3)
    assert res["f_full"] == pytest.approx(best, rel=1e-6)
    # with small samples the result is a sample solution: never below the optimum
    res = bigmeans.bigmeans(x[:, None], 2, dict(s_min=100, s_max=400, workers=4, passes=5),
                            BUDGET, seed=3)
    assert best * (1 - 1e-6) <= res["f_full"] <= best * 1.01


def test_incumbent_rules_and_s_opt():
    X = (np.random.default_rng(12).standard_normal((3000, 3)) * 2).astype(np.float32)
    X[:1000] += 9
    X[1000:2000] -= 9
    pol = dict(s_min=100, s_max=900, workers=4, passes=5)
    res = bigmeans.bigmeans(X, 4, pol, dict(BUDGET, rounds=3, eval_full_each_round=True), seed=5)
    log = res["log"]
    for w in range(4):
        tr = log["fhat_trace"][w]
        for a, b in zip(tr, tr[1:]):
            if b[0] == "pass":             # passes never raise f_hat within a round
                assert b[2] <= a[2]
    inc = [e[3] for e in log["incumbent"]]
    assert all(b <= a for a, b in zip(inc, inc[1:]))
    drawn = {s for w in range(4) for s in log["sizes"][w]}
    assert set(res["L"]) <= drawn
    assert sum(sum(a) for a in log["accepts"]) == len(res["L"])
    L = res["L"]
    assert res["s_opt"] == int(np.floor(np.mean(L) + 0.5))
    assert res["best_worker"] == int(np.argmin(res["f_hat"]))


def test_single_worker_full_sample_is_kmeanspp_then_lloyd():
    X = np.random.default_rng(13).standard_normal((500, 2)).astype(np.float32) * 3
    k, seed = 4, 21
    res = bigmeans.bigmeans(X, k, dict(s_min=500, s_max=500, workers=1, passes=1),
                            dict(BUDGET, rounds=1), seed=seed)
    idx = bigmeans.sample_indices(seed, rng.P_PASS, 0, 0, 0, 500, 500)
    C0, _ = kmeans.kmeanspp_reseed(X[idx], np.zeros((k, 2), np.float32), np.ones(k, bool),
                                   rng.stream_key(seed, rng.P_KPP, 0, 0, 0))
    ll = kmeans.lloyd(X[idx], C0)
    assert np.array_equal(res["C"], ll["C"])
    assert res["f_full"] == ll["f"]            # same point set, other order: exact sums agree
    assert res["L"] == [500]


def test_deterministic_and_seed_sensitive():
    X = np.random.default_rng(14).standard_normal((2000, 2)).astype(np.float32) * 4
    pol = dict(set=[100, 200, 400], workers=3, passes=3)
    a = bigmeans.bigmeans(X, 3, pol, BUDGET, seed=1)
    b = bigmeans.bigmeans(X, 3, pol, BUDGET, seed=1)
    c = bigmeans.bigmeans(X, 3, pol, BUDGET, seed=2)
    assert np.array_equal(a["C"], b["C"]) and a["f_full"] == b["f_full"]
    assert a["L"] == b["L"]
    assert a["L"] != c["L"] or not np.array_equal(a["C"], c["C"])
