"""Counter-based random numbers for the oracle (test infrastructure only).

Philox4x64-10 is written here from its published definition (Salmon, Moraes,
Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4-word
64-bit counter and a 2-word key, ten rounds of two 64x64->128 multiplies with
the key bumped by two Weyl constants between rounds.

Every random choice the method makes (the sample size s_w of Algorithm 1, the
uniform sample of Sec. 4.1, the K-means++ draws) is keyed by the purpose and
by (worker, round, pass), so a draw never depends on execution order.  The
stream layout, shared by contract with the CUDA library (which has its own,
independent implementation), is:

    key[0] = seed
    key[1] = purpose << 56 | worker << 40 | round << 16 | pass
    counter = (c0, c1, 0, 0) -- c0 = draw index, c1 = sub-stream (e.g. centroid)

Bounded integers use Lemire's multiply-and-reject method (Lemire, "Fast random
integer generation in an interval", ACM TOMACS 2019): word w is accepted when
the low half of w*bound is >= (2^64 - bound) mod bound; the draw is the high
half.  One counter block supplies four candidate words; if all four are
rejected (probability below (bound/2^64)^4) the high half of the last word is
used.
"""
import numpy as np

M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
M32 = np.uint64(0xFFFFFFFF)
PHILOX_M0 = np.uint64(0xD2E7470EE14C6C93)
PHILOX_M1 = np.uint64(0xCA5A826395121157)
PHILOX_W0 = np.uint64(0x9E3779B97F4A7C15)
PHILOX_W1 = np.uint64(0xBB67AE8584CAA73B)

# purposes (high byte of key[1])
P_SIZE = 1     # s_w drawn in [s_min, s_max] each round        (Alg. 1)
P_EVAL = 2     # fresh sample used to recompute f_hat_w        (Alg. 1, Sec. 4.3)
P_PASS = 3     # the sample S_w of one pass                    (Alg. 1, Sec. 4.1)
P_KPP = 4      # K-means++ draws while re-seeding              (Sec. 4.1, Sec. 5)
P_FINAL = 5    # the common sample of size s_opt               (Alg. 1)


def _u64(a):
    return np.asarray(a, dtype=np.uint64)


def mulhilo64(a, b):
    """Full 128-bit product of uint64 arrays, returned as (hi, lo)."""
    a = _u64(a)
    b = _u64(b)
    a_lo, a_hi = a & M32, a >> np.uint64(32)
    b_lo, b_hi = b & M32, b >> np.uint64(32)
    p0 = a_lo * b_lo
    p1 = a_lo * b_hi
    p2 = a_hi * b_lo
    p3 = a_hi * b_hi
    mid = (p0 >> np.uint64(32)) + (p1 & M32) + (p2 & M32)
    hi = p3 + (p1 >> np.uint64(32)) + (p2 >> np.uint64(32)) + (mid >> np.uint64(32))
    with np.errstate(over="ignore"):
        lo = a * b
    return hi, lo


def philox4x64(counter, key, rounds=10):
    """Philox4x64-R.  counter: (..., 4) uint64, key: (2,) or (..., 2) uint64.

    Returns an (..., 4) uint64 array."""
    ctr = _u64(counter)
    k = np.broadcast_to(_u64(key), ctr.shape[:-1] + (2,))
    x0, x1, x2, x3 = (ctr[..., i].copy() for i in range(4))
    k0 = k[..., 0].copy()
    k1 = k[..., 1].copy()
    with np.errstate(over="ignore"):
        for r in range(rounds):
            if r:
                k0 = k0 + PHILOX_W0
                k1 = k1 + PHILOX_W1
            hi0, lo0 = mulhilo64(PHILOX_M0, x0)
            hi1, lo1 = mulhilo64(PHILOX_M1, x2)
            x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return np.stack([x0, x1, x2, x3], axis=-1)


def stream_key(seed, purpose, worker=0, rnd=0, pss=0):
    """The 2-word Philox key of one (purpose, worker, round, pass) stream."""
    assert 0 <= worker < (1 << 16) and 0 <= rnd < (1 << 24) and 0 <= pss < (1 << 16)
    k1 = (int(purpose) << 56) | (int(worker) << 40) | (int(rnd) << 16) | int(pss)
    return np.array([int(seed) & 0xFFFFFFFFFFFFFFFF, k1], dtype=np.uint64)


def blocks(key, c0, c1=0):
    """Philox blocks for counters (c0[i], c1, 0, 0); c0 may be an array."""
    c0 = np.atleast_1d(_u64(c0))
    ctr = np.zeros(c0.shape + (4,), dtype=np.uint64)
    ctr[..., 0] = c0
    ctr[..., 1] = np.uint64(c1)
    return philox4x64(ctr, key)


def uniform_below(blk, bound):
    """Lemire draw in [0, bound) from each 4-word block; returns int64 array."""
    bound = int(bound)
    assert 1 <= bound < (1 << 63)
    b = np.uint64(bound)
    with np.errstate(over="ignore"):
        thr = np.uint64((-bound) % (1 << 64) % bound)
    hi, lo = mulhilo64(blk, b)              # (..., 4)
    ok = lo >= thr
    first = np.argmax(ok, axis=-1)          # index of first accepted word
    anyok = ok.any(axis=-1)
    first = np.where(anyok, first, 3)
    out = np.take_along_axis(hi, first[..., None], axis=-1)[..., 0]
    return out.astype(np.int64)


def draw_below(key, c0, c1, bound):
    """One bounded draw from counter (c0, c1, 0, 0)."""
    return int(uniform_below(blocks(key, c0, c1), bound)[0])
