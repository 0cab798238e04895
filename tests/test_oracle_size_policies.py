"""Pins of the sample-size policies of the oracle (Alg. 1's size draw and
the exploration / exploitation variants the paper names as future work).

* kind 0 is the paper's uniform integer draw on [s_min, s_max], unchanged;
* kind 1 (octave-uniform) puts probability 1/O on each octave
  [s_min 2^i, s_min 2^(i+1) - 1] (the last one ending at s_max) and is
  uniform inside each octave -- checked with chi-square tests;
* exploit uses the mean of L before the round, rounded half up and clipped,
  with the stated probability, and never before L has an entry.
"""
import numpy as np
import pytest

from oracle import bigmeans as obm
from oracle import rng as orng

scipy_stats = pytest.importorskip("scipy.stats")


def _sizes(policy, n=8000, seed=77, L_sum=0, L_len=0):
    return np.array([obm.draw_size(seed, w, r, policy, L_sum, L_len)
                     for w in range(100) for r in range(n // 100)])


def test_uniform_kind_is_the_papers_draw():
    pol = dict(s_min=1000, s_max=64000)
    for w, r in [(0, 0), (3, 7), (15, 1)]:
        key = orng.stream_key(5, orng.P_SIZE, w, r, 0)
        assert obm.draw_size(5, w, r, pol) == 1000 + orng.draw_below(key, 0, 0, 63001)


def test_octave_uniform_octaves_and_values():
    pol = dict(s_min=3, s_max=40, kind=1)          # octaves [3,5] [6,11] [12,23] [24,40]
    s = _sizes(pol)
    assert s.min() >= 3 and s.max() <= 40
    edges = [(3, 5), (6, 11), (12, 23), (24, 40)]
    counts = [int(((s >= a) & (s <= b)).sum()) for a, b in edges]
    assert sum(counts) == s.size
    assert scipy_stats.chisquare(counts).pvalue > 1e-3
    for a, b in edges:                               # uniform inside each octave
        inside = s[(s >= a) & (s <= b)]
        c = np.bincount(inside - a, minlength=b - a + 1)
        assert scipy_stats.chisquare(c).pvalue > 1e-3


def test_octave_uniform_degenerate_ranges():
    assert set(_sizes(dict(s_min=7, s_max=7, kind=1), n=300)) == {7}
    s = _sizes(dict(s_min=5, s_max=9, kind=1), n=3000)    # one octave [5, 9]
    assert set(s) == {5, 6, 7, 8, 9}


def test_exploit_uses_the_rounded_mean_of_L():
    pol = dict(s_min=100, s_max=5000, exploit=100)
    assert obm.draw_size(1, 0, 3, pol, L_sum=7, L_len=2) == 100          # mean 4 clipped up
    assert obm.draw_size(1, 0, 3, pol, L_sum=2001 + 2002, L_len=2) == 2002   # 2001.5 rounds up
    assert obm.draw_size(1, 0, 3, pol, L_sum=10 ** 6, L_len=1) == 5000       # clipped down
    # no L yet: the base draw
    base = obm.draw_size(1, 0, 3, dict(s_min=100, s_max=5000))
    assert obm.draw_size(1, 0, 3, pol, 0, 0) == base


def test_exploit_probability():
    pol = dict(s_min=1000, s_max=64000, exploit=30)
    s = _sizes(pol, n=8000, L_sum=12345 * 3, L_len=3)
    frac = float((s == 12345).mean())
    # 30% exploitation plus the base draw hitting 12345 by chance (1 / 63001)
    assert abs(frac - 0.30) < 4 * np.sqrt(0.3 * 0.7 / s.size)


def test_fit_with_exploit_draws_from_L_of_previous_rounds():
    X = np.random.default_rng(0).normal(size=(3000, 2)).astype(np.float32)
    pol = dict(s_min=100, s_max=2000, workers=3, passes=2, exploit=100)
    out = obm.bigmeans(X, 3, pol, dict(rounds=3), seed=4)
    sizes = out["log"]["sizes"]
    # round 0: L empty, base draws; later rounds: every worker takes the mean of L so far
    L_by_round, L = [], []
    for t in range(3):
        L_by_round.append(list(L))
        for w in range(3):
            for p in range(2):
                if out["log"]["accepts"][w][t * 2 + p]:
                    L.append(sizes[w][t])
    for t in (1, 2):
        Lt = L_by_round[t]
        want = (2 * sum(Lt) + len(Lt)) // (2 * len(Lt))
        assert all(sizes[w][t] == min(max(want, 100), 2000) for w in range(3))
