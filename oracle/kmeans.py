"""Oracle K-means pieces of Big-means (test infrastructure only).

Written from arXiv 2403.18766: Eq. (1) (the MSSC objective f(C, X)),
Sec. 4.1 (K-means on a sample, K-means++ for the first sample and for
degenerate clusters), Sec. 5 (Lloyd stops after 300 iterations or at a
relative tolerance of 1e-4; K-means++ draws three candidate points).

Two numeric modes.

``exact32`` (the mode the CUDA path must reproduce bit for bit).  The paper
fixes no precision, so per-point decisions are taken in FP32, the precision
the kernels compute in, with one fixed operation order; every sum that feeds a
decision is exact:

* d32(x, c): t = fl32(x_d - c_d), acc = fl32(acc + fl32(t*t)) over ascending
  d, no fused multiply-add.
* label(x) = argmin_j d32(x, c_j), lowest j on ties.
* f(C, P) = RN64( exact sum over x in P of d32(x, c_label(x)) )  -- Eq. (1).
* centroid update c_j = RN32( RN64(exact sum of members) / count_j ); a
  cluster with no members keeps its centroid and is "degenerate".
* K-means++ weights are D^2 in FP32 quantised to integers on a grid set by the
  current maximum: w_i = floor(D2_i * 2^(31 - E)), where max D2 = f * 2^E,
  f in [0.5, 1).  Candidate potentials use the same grid and integer sums.

``pure64``: the same algorithm with FP64 distances and FP64 centroids, used
to report how far exact32 results sit from an all-FP64 computation.

Exact sums use ``math.fsum``, which returns the correctly rounded value of the
exact sum of its float64 inputs; every FP32 value is exact in float64.
"""
import math

import numpy as np

from . import rng

MODES = ("exact32", "pure64")


# ----------------------------------------------------------------- distances
def d32_all(S, C):
    """d32(S_i, C_j) for all i, j as an (s, k) float32 array (exact32)."""
    S = np.asarray(S, dtype=np.float32)
    C = np.asarray(C, dtype=np.float32)
    s, n = S.shape
    acc = np.zeros((s, C.shape[0]), dtype=np.float32)
    for d in range(n):
        t = S[:, d][:, None] - C[:, d][None, :]
        acc = acc + t * t
    return acc


def d64_all(S, C):
    """FP64 squared distances (pure64)."""
    S = np.asarray(S, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    acc = np.zeros((S.shape[0], C.shape[0]), dtype=np.float64)
    for d in range(S.shape[1]):
        t = S[:, d][:, None] - C[:, d][None, :]
        acc = acc + t * t
    return acc


def d32_rows(S, c):
    """d32(S_i, c) for one centroid c, as a length-s float32 vector."""
    return d32_all(S, np.asarray(c, dtype=np.float32)[None, :])[:, 0]


def exact_sum(values):
    """RN64 of the exact sum of the given (float32 or float64) values."""
    return math.fsum(np.asarray(values, dtype=np.float64).tolist())


# ------------------------------------------------------ assignment / Eq. (1)
def assign(S, C, mode="exact32", chunk=1 << 16):
    """Nearest-centroid labels (lowest index on ties) and per-point distance.

    Implements the inner min of Eq. (1).  Returns (labels int32, dist)."""
    S = np.asarray(S)
    labels = np.empty(S.shape[0], dtype=np.int32)
    dist = np.empty(S.shape[0], dtype=np.float32 if mode == "exact32" else np.float64)
    for a in range(0, S.shape[0], chunk):
        D = d32_all(S[a:a + chunk], C) if mode == "exact32" else d64_all(S[a:a + chunk], C)
        lab = np.argmin(D, axis=1)          # first minimum = lowest index on ties
        labels[a:a + chunk] = lab
        dist[a:a + chunk] = D[np.arange(D.shape[0]), lab]
    return labels, dist


def objective(S, C, mode="exact32"):
    """f(C, S) of Eq. (1): exact sum of nearest-centroid distances, rounded once."""
    _, dist = assign(S, C, mode)
    return exact_sum(dist)


# --------------------------------------------------------------- Lloyd (A2)
def update_centroids(S, labels, C, mode="exact32"):
    """Centroid = mean of its members (exact sum, one FP64 division).

    exact32 rounds the mean to FP32.  Returns (C_new, counts)."""
    S = np.asarray(S)
    k, n = C.shape
    counts = np.bincount(labels, minlength=k).astype(np.int64)
    C_new = np.array(C, dtype=np.float32 if mode == "exact32" else np.float64, copy=True)
    order = np.argsort(labels, kind="stable")
    bounds = np.concatenate([[0], np.cumsum(counts)])
    for j in range(k):
        if counts[j] == 0:
            continue                                   # empty: keep old centroid
        rows = S[order[bounds[j]:bounds[j + 1]]]
        for d in range(n):
            sm = exact_sum(rows[:, d])
            mean = sm / float(counts[j])               # IEEE FP64 division
            C_new[j, d] = np.float32(mean) if mode == "exact32" else mean
    return C_new, counts


def lloyd(S, C0, max_iter=300, tol=1e-4, mode="exact32"):
    """Lloyd's K-means on sample S from initial centroids C0 (Sec. 4.1, Sec. 5).

    One iteration = centroid update followed by re-assignment.  The run stops
    after ``max_iter`` updates, or as soon as the objective of the new
    assignment improved by no more than ``tol`` times the previous objective
    (f_prev - f_new <= tol * f_prev, FP64).  The returned f is f(C, S) of the
    returned centroids; ``empty`` marks clusters with no member in that final
    assignment (the degenerate clusters of Sec. 4.1).

    Returns dict(C, f, iters, empty, trace) where trace lists every f."""
    C = np.array(C0, dtype=np.float32 if mode == "exact32" else np.float64, copy=True)
    labels, dist = assign(S, C, mode)
    f = exact_sum(dist)
    trace = [f]
    iters = 0
    while iters < max_iter:
        C, _ = update_centroids(S, labels, C, mode)
        iters += 1
        labels, dist = assign(S, C, mode)
        f_new = exact_sum(dist)
        trace.append(f_new)
        stop = (f - f_new) <= tol * f
        f = f_new
        if stop:
            break
    counts = np.bincount(labels, minlength=C.shape[0])
    return dict(C=C, f=f, iters=iters, empty=counts == 0, trace=trace, labels=labels)


# ---------------------------------------------------- K-means++ (A3, A4)
def quantise(D2, E):
    """floor(D2 * 2^(31-E)) as int64, D2 in float32 (exact in float64)."""
    return np.floor(np.ldexp(np.asarray(D2, dtype=np.float64), 31 - E)).astype(np.int64)


def kmeanspp_reseed(S, C, degenerate, key, n_trials=3, mode="exact32"):
    """Re-initialise the degenerate centroids of C with greedy K-means++ on S.

    Sec. 4.1: the first sample is seeded with K-means++ and afterwards only
    degenerate clusters are re-initialised; Sec. 5: K-means++ uses three
    candidate points.  Degenerate centroids are re-seeded in increasing index
    order; non-degenerate and already re-seeded centroids count as chosen.

    * No centroid chosen yet: the centroid is the sample point at a uniform
      index, draw (0, j) of ``key``.
    * Otherwise D2_i = min over chosen c of d(S_i, c).  Candidate l in
      0..n_trials-1 is the first i whose integer prefix sum of the weights
      exceeds u_l, u_l uniform in [0, W) from draw (l, j), W = sum of weights.
      The kept candidate has the least potential sum_i q(min(D2_i, d(S_i,
      cand))) (lowest l on ties).  If every D2 is zero, the centroid is the
      point at uniform index (0, j).

    Returns (C_new, chosen_indices)."""
    S = np.asarray(S, dtype=np.float32 if mode == "exact32" else np.float64)
    s = S.shape[0]
    C = np.array(C, dtype=S.dtype, copy=True)
    k = C.shape[0]
    live = ~np.asarray(degenerate, dtype=bool)
    dist_rows = d32_rows if mode == "exact32" else (
        lambda X, c: d64_all(X, np.asarray(c, dtype=np.float64)[None, :])[:, 0])
    D2 = None
    if live.any():
        D2 = np.min(d32_all(S, C[live]) if mode == "exact32" else d64_all(S, C[live]), axis=1)
    picks = {}
    for j in range(k):
        if live[j]:
            continue
        if D2 is None:
            idx = rng.draw_below(key, 0, j, s)
        else:
            M = float(D2.max())
            if M == 0.0:
                idx = rng.draw_below(key, 0, j, s)
            else:
                E = math.frexp(M)[1]
                w = quantise(D2, E)
                prefix = np.cumsum(w)
                W = int(prefix[-1])
                best = None
                for l in range(n_trials):
                    u = rng.draw_below(key, l, j, W)
                    cand = int(np.searchsorted(prefix, u, side="right"))
                    phi = int(quantise(np.minimum(D2, dist_rows(S, S[cand])), E).sum())
                    if best is None or phi < best[0]:
                        best = (phi, cand)
                idx = best[1]
        C[j] = S[idx]
        picks[j] = idx
        live[j] = True
        dj = dist_rows(S, C[j])
        D2 = dj if D2 is None else np.minimum(D2, dj)
    return C, picks
