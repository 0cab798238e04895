"""Oracle for Algorithm 1 of arXiv 2403.18766 (test infrastructure only).

Competitive stochastic sample size Big-means, restated step by step from
Algorithm 1 and its description (Sec. 4.2, Sec. 4.3), with the settings of
Sec. 5.  Readings of points the paper leaves open:

* the uniform sample is drawn without replacement: bounded draws r_0, r_1, ...
  in [0, m) are taken in counter order and repeats are skipped until s
  distinct indices are collected; the sample keeps that order;
* "Recalculate f_hat_w with the new s_w" uses a fresh sample of size s_w
  (purpose EVAL), and is skipped while every centroid of w is degenerate
  (f_hat_w stays +inf);
* K-means++ re-seeding overwrites the degenerate centroids of C_w in place,
  as the pseudocode does, whether or not the pass is then accepted; the
  degenerate set changes only on acceptance (empty clusters of C_new);
* s_opt is the mean of L rounded half up (Sec. 4.2: "a simple mean"), clipped
  to the size range; if L is empty s_opt = s_max;
* the common recheck draws one sample S (purpose FINAL) shared by all
  workers; the least f_hat_w wins, lowest w on ties.
"""
import numpy as np

from . import kmeans, rng


def sample_indices(seed, purpose, worker, rnd, pss, m, s):
    """First s distinct bounded draws in [0, m), in order of first occurrence."""
    m, s = int(m), int(s)
    assert 0 <= s <= m
    if s == 0:
        return np.zeros(0, dtype=np.int64)
    key = rng.stream_key(seed, purpose, worker, rnd, pss)
    T = s + (s * s) // m + 64
    while True:
        draws = rng.uniform_below(rng.blocks(key, np.arange(T, dtype=np.uint64)), m)
        _, first = np.unique(draws, return_index=True)
        if first.size >= s:
            keep = np.sort(first)[:s]
            return draws[keep]
        T *= 2


def draw_size(seed, worker, rnd, policy, L_sum=0, L_len=0):
    """s_w for (worker, round), from the size stream (SIZE, worker, round, 0).

    The paper (Alg. 1): a uniform integer in [s_min, s_max], or uniform over
    a configured set.  The future-work variants (Sec. 7 proposes trying
    further ways of exploring the size range and of reusing the best size
    found so far):
      kind 1  - octave-uniform: octave i uniform in [0, O) with O the least
                t >= 1 with s_min * 2^t >= s_max (O = 1 when s_min = s_max),
                then uniform inside [s_min 2^i, s_min 2^(i+1) - 1]; the last
                octave ends at s_max;
      exploit - with probability exploit/100 (draw (1, 0) below 100 less
                than exploit), the mean of L before this round, rounded half
                up and clipped to the size range, when L is not empty.
    Draw (0, 0) picks the set entry, the value or the octave; draw (2, 0) the
    value inside the octave."""
    key = rng.stream_key(seed, rng.P_SIZE, worker, rnd, 0)
    exploit = int(policy.get("exploit", 0))
    if exploit > 0 and L_len > 0 and rng.draw_below(key, 1, 0, 100) < exploit:
        lo, hi = size_range(policy, 1 << 62)
        v = (2 * L_sum + L_len) // (2 * L_len)
        return int(min(max(v, lo), hi))
    if policy.get("set"):
        vals = list(policy["set"])
        return int(vals[rng.draw_below(key, 0, 0, len(vals))])
    lo, hi = int(policy["s_min"]), int(policy["s_max"])
    if int(policy.get("kind", 0)) == 1:
        t = 0
        while lo * 2 ** t < hi:
            t += 1
        octaves = max(1, t)
        i = rng.draw_below(key, 0, 0, octaves)
        a = lo * 2 ** i
        b = hi if i == octaves - 1 else lo * 2 ** (i + 1) - 1
        return a + rng.draw_below(key, 2, 0, b - a + 1)
    return lo + rng.draw_below(key, 0, 0, hi - lo + 1)


def size_range(policy, m):
    if policy.get("set"):
        vals = [min(int(v), m) for v in policy["set"]]
        return min(vals), max(vals)
    return int(policy["s_min"]), min(int(policy["s_max"]), m)


def normalise_policy(policy, m):
    p = dict(policy)
    if p.get("set"):
        p["set"] = [min(int(v), m) for v in p["set"]]
    else:
        p["s_max"] = min(int(p["s_max"]), m)      # Sec. 5: s_max = min(2s, m)
    return p


def bigmeans(X, k, policy, budget, seed, mode="exact32"):
    """Run Algorithm 1 with a round-count budget.

    policy: dict(s_min, s_max) or dict(set=[...]); plus workers (W) and
            passes (p).
    budget: dict(rounds=T, max_lloyd=300, tol=1e-4, kpp_candidates=3,
            eval_full_each_round=False).
    Returns a dict with C (k x n), labels (m), f_full, s_opt, L, f_hat (final
    recheck values), best_worker, per-worker state and traces."""
    X = np.asarray(X, dtype=np.float32)
    m, n = X.shape
    W = int(policy["workers"])
    P = int(policy.get("passes", 10))
    T = int(budget["rounds"])
    max_lloyd = int(budget.get("max_lloyd", 300))
    tol = float(budget.get("tol", 1e-4))
    L_trials = int(budget.get("kpp_candidates", 3))
    policy = normalise_policy(policy, m)
    s_lo, s_hi = size_range(policy, m)
    cdt = np.float32 if mode == "exact32" else np.float64

    # Initialisation (Alg. 1): all centroids degenerate, f_hat = inf, t = 0, L empty
    C = [np.zeros((k, n), dtype=cdt) for _ in range(W)]
    deg = [np.ones(k, dtype=bool) for _ in range(W)]
    fhat = [np.inf] * W
    L = []
    log = dict(lloyd_iters=0, pts_k=0, passes=0, accepts=[[] for _ in range(W)],
               fhat_trace=[[] for _ in range(W)], incumbent=[], sizes=[[] for _ in range(W)])
    inc_f = np.inf

    for t in range(T):
        L_sum, L_len = sum(L), len(L)                        # L as it stood before the round
        for w in range(W):
            s_w = draw_size(seed, w, t, policy, L_sum, L_len)
            log["sizes"][w].append(s_w)
            if not deg[w].all():                             # recompute f_hat_w with new s_w
                idx = sample_indices(seed, rng.P_EVAL, w, t, 0, m, s_w)
                fhat[w] = kmeans.objective(X[idx], C[w], mode)
            log["fhat_trace"][w].append(("eval", t, fhat[w]))
            for p in range(P):
                idx = sample_indices(seed, rng.P_PASS, w, t, p, m, s_w)
                S = X[idx]
                if deg[w].any():
                    key = rng.stream_key(seed, rng.P_KPP, w, t, p)
                    C[w], _ = kmeans.kmeanspp_reseed(S, C[w], deg[w], key, L_trials, mode)
                res = kmeans.lloyd(S, C[w], max_lloyd, tol, mode)
                log["lloyd_iters"] += res["iters"]
                log["pts_k"] += s_w * k * (res["iters"] + 1)   # assignment passes
                log["passes"] += 1
                accepted = res["f"] < fhat[w]
                if accepted:
                    C[w] = res["C"]
                    deg[w] = res["empty"].copy()
                    fhat[w] = res["f"]
                    L.append(s_w)
                log["accepts"][w].append(bool(accepted))
                log["fhat_trace"][w].append(("pass", t, fhat[w]))
        if budget.get("eval_full_each_round"):
            wb = int(np.argmin(fhat))
            F = kmeans.objective(X, C[wb], mode)
            inc_f = min(inc_f, F)
            log["incumbent"].append((t, wb, F, inc_f))

    # s_opt = mean of L (Sec. 4.2), rounded half up
    if L:
        s_opt = (2 * sum(L) + len(L)) // (2 * len(L))
        s_opt = min(max(s_opt, s_lo), s_hi)
    else:
        s_opt = s_hi
    idx = sample_indices(seed, rng.P_FINAL, 0, 0, 0, m, s_opt)
    S = X[idx]
    f_final = [kmeans.objective(S, C[w], mode) for w in range(W)]
    best = int(np.argmin(f_final))                          # lowest w on ties
    C_best = C[best]
    labels, dist = kmeans.assign(X, C_best, mode)
    f_full = kmeans.exact_sum(dist)
    return dict(C=C_best, labels=labels, f_full=f_full, s_opt=int(s_opt), L=L,
                f_hat=f_final, best_worker=best, C_workers=C, deg=deg,
                fhat_rounds=fhat, log=log)
