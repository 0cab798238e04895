"""Pins for the oracle's random streams (Philox4x64-10, bounded draws, samples).

The oracle's Philox is checked against numpy's independent Philox bit
generator and the published known-answer vectors; the bounded draw against
its closed form for power-of-two bounds and against the rejection rule written
with Python integers; the sampler against a plain sequential loop and against
uniformity statistics.
"""
import os
from collections import Counter

import numpy as np
import pytest
from scipy import stats

from oracle import bigmeans, rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_matches_numpy_bit_generator():
    # numpy's Philox is Philox4x64-10; it increments its counter before each block.
    for key in ([0, 0], [12345, 0xDEADBEEF], [2**64 - 1, 7]):
        key = np.array(key, dtype=np.uint64)
        bg = np.random.Philox(key=key, counter=np.zeros(4, dtype=np.uint64))
        raw = bg.random_raw(4 * 64)
        ctr = np.zeros((64, 4), dtype=np.uint64)
        ctr[:, 0] = np.arange(1, 65, dtype=np.uint64)
        mine = rng.philox4x64(ctr, key).reshape(-1)
        assert np.array_equal(raw, mine)


def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x64_10_kat.txt")) as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        ctr = np.array(v[0:4], dtype=np.uint64)
        key = np.array(v[4:6], dtype=np.uint64)
        assert [int(x) for x in rng.philox4x64(ctr, key)] == v[6:10]


def test_mulhilo_against_python_ints():
    g = np.random.default_rng(1)
    a = g.integers(0, 2**63, 1000, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    b = g.integers(0, 2**63, 1000, dtype=np.uint64)
    hi, lo = rng.mulhilo64(a, b)
    for x, y, h, l in zip(a.tolist(), b.tolist(), hi.tolist(), lo.tolist()):
        p = x * y
        assert h == p >> 64 and l == p & (2**64 - 1)


def test_uniform_below_power_of_two_is_top_bits():
    key = rng.stream_key(3, rng.P_PASS, 1, 2, 3)
    blk = rng.blocks(key, np.arange(500, dtype=np.uint64))
    for bits in (1, 7, 20, 40):
        got = rng.uniform_below(blk, 1 << bits)
        want = (blk[:, 0] >> np.uint64(64 - bits)).astype(np.int64)
        assert np.array_equal(got, want)


def test_uniform_below_rejection_rule_with_python_ints():
    # A bound just above 2^62 rejects about a quarter of all words, so the
    # four-word fallback is exercised too.
    bound = (1 << 62) + 12345
    key = rng.stream_key(9, rng.P_KPP, 0, 0, 0)
    blk = rng.blocks(key, np.arange(400, dtype=np.uint64))
    got = rng.uniform_below(blk, bound)
    thr = (2**64 - bound) % bound
    for words, g in zip(blk.tolist(), got.tolist()):
        want = None
        for w in words:
            p = w * bound
            if p & (2**64 - 1) >= thr:
                want = p >> 64
                break
        if want is None:
            want = (words[3] * bound) >> 64
        assert g == want


def test_uniform_below_chi_square():
    key = rng.stream_key(5, rng.P_SIZE, 0, 0, 0)
    x = rng.uniform_below(rng.blocks(key, np.arange(60000, dtype=np.uint64)), 12)
    counts = np.bincount(x, minlength=12)
    assert stats.chisquare(counts).pvalue > 1e-4


def _sample_by_loop(seed, purpose, w, t, p, m, s):
    key = rng.stream_key(seed, purpose, w, t, p)
    out, seen, c = [], set(), 0
    while len(out) < s:
        r = rng.draw_below(key, c, 0, m)
        c += 1
        if r not in seen:
            seen.add(r)
            out.append(r)
    return out


@pytest.mark.parametrize("m,s", [(50, 1), (50, 17), (50, 50), (1000, 600), (10_000, 2000)])
def test_sample_is_first_distinct_draws(m, s):
    got = bigmeans.sample_indices(11, rng.P_PASS, 2, 1, 4, m, s)
    assert got.tolist() == _sample_by_loop(11, rng.P_PASS, 2, 1, 4, m, s)
    assert len(set(got.tolist())) == s and got.min() >= 0 and got.max() < m


def test_sample_full_size_is_permutation():
    got = bigmeans.sample_indices(1, rng.P_FINAL, 0, 0, 0, 300, 300)
    assert sorted(got.tolist()) == list(range(300))


def test_sample_inclusion_is_uniform():
    m, s, reps = 40, 10, 3000
    inc = Counter()
    for r in range(reps):
        inc.update(bigmeans.sample_indices(r, rng.P_EVAL, 0, 0, 0, m, s).tolist())
    counts = np.array([inc[i] for i in range(m)])
    assert counts.sum() == s * reps
    assert stats.chisquare(counts).pvalue > 1e-4


def test_streams_are_distinct():
    a = bigmeans.sample_indices(1, rng.P_PASS, 0, 0, 0, 10**6, 100)
    b = bigmeans.sample_indices(1, rng.P_PASS, 0, 0, 1, 10**6, 100)
    c = bigmeans.sample_indices(1, rng.P_EVAL, 0, 0, 0, 10**6, 100)
    d = bigmeans.sample_indices(2, rng.P_PASS, 0, 0, 0, 10**6, 100)
    assert len({tuple(a), tuple(b), tuple(c), tuple(d)}) == 4
