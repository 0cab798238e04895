"""A competitive Big-means fit sharded over ranks (one GPU per rank, X replicated).

Algorithm 1's workers are independent until the end (Sec. 4.2-4.3): they
share only the list L of improving sample sizes, whose mean is s_opt, and the
final common recheck, whose least f_hat_w picks the result.  So rank r of R
runs the workers [W r / R, W (r + 1) / R) of a W-worker fit with the library
(bm_fit_set_workers) and the ranks exchange, on the host, through any
torch.distributed process group (NCCL between GPUs, gloo on CPU):

1. every rank's (sum of L, |L|) -- an all-gather of two integers per rank;
   s_opt = the mean of the global L rounded half up, clipped to the size
   range (s_max if L is empty);
2. each rank's least (f_hat_w, w) on the common sample of size s_opt (the
   same draws on every rank) -- an all-gather of one pair per rank; the least
   f, lowest w on ties, is w*;
3. the centroids of w*, broadcast from the rank that holds it; the full-data
   pass then gives the labels and f(C, X).

The result equals the unsharded fit's bit for bit.  This module moves only
small host values between ranks; all arithmetic of the method runs in the
library.  `group` is a torch.distributed process group (None: the default
group), or False for a single process that holds every worker (no
collective).
"""
import torch


def worker_range(W, rank, world):
    """The workers [w_begin, w_end) of `rank` out of `world` ranks."""
    return W * rank // world, W * (rank + 1) // world


def size_range(policy, m):
    """(s_lo, s_hi) of a policy dict, s_max and set entries clipped to m (Sec. 5)."""
    if policy.get("set"):
        vals = [min(int(v), m) for v in policy["set"]]
        return min(vals), max(vals)
    return int(policy["s_min"]), min(int(policy["s_max"]), m)


def s_opt_from(L_sum, L_len, s_lo, s_hi):
    """Mean of L rounded half up, clipped to the size range; s_hi if L is empty."""
    if L_len == 0:
        return s_hi
    return min(max((2 * L_sum + L_len) // (2 * L_len), s_lo), s_hi)


def _all_gather(values, group, device):
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64 if any(isinstance(v, float) for v in values) else torch.int64,
                     device=device)
    out = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(out, t, group=group)
    return [o.tolist() for o in out]


def global_L(L_sum, L_len, group=None, device="cpu"):
    """Sum of every rank's (sum of L, |L|)."""
    if group is False:
        return int(L_sum), int(L_len)
    parts = _all_gather([int(L_sum), int(L_len)], group, device)
    return sum(p[0] for p in parts), sum(p[1] for p in parts)


def least(pairs):
    """The least (f, w) of a list of pairs: least f, lowest w on ties."""
    return min(pairs, key=lambda p: (p[0], p[1]))


def pick_best(f_local, w_begin, group=None, device="cpu"):
    """The global least (f_hat_w, w) from each rank's list of f_hat for its
    workers w_begin, w_begin + 1, ...; returns (f, w)."""
    f, w = least([(float(v), w_begin + i) for i, v in enumerate(f_local)])
    if group is False:
        return f, w
    parts = _all_gather([f, float(w)], group, device)
    f, w = least([(p[0], int(p[1])) for p in parts])
    return f, int(w)


def broadcast_centroids(C, owner, shape, group=None, device="cpu"):
    """C (k x n float32) of the owner rank on every rank."""
    import torch.distributed as dist
    import numpy as np
    if group is False:
        return C
    if C is None:
        buf = torch.empty(shape, dtype=torch.float32, device=device)
    else:
        buf = torch.as_tensor(np.ascontiguousarray(C) if not isinstance(C, torch.Tensor) else C,
                              dtype=torch.float32).to(device).contiguous()
    dist.broadcast(buf, src=owner, group=group)
    return buf


def fit_sharded(Xd, k, policy, budget, seed, rank, world, group=None, comm_device=None, stream=None):
    """Rank `rank`'s part of one fit over `world` ranks: its workers' rounds
    on this GPU, then the three exchanges and the full-data pass.  policy and
    budget are dicts (as for native.make_policy / make_budget; no exploit
    policy).  Returns (C, labels, info) on every rank."""
    from . import native
    m = Xd.shape[0]
    comm_device = comm_device or Xd.device
    W = int(policy["workers"])
    w0, w1 = worker_range(W, rank, world)
    sess = native.FitSession(Xd, k, native.make_policy(**policy), native.make_budget(**budget), seed=seed,
                             stream=stream)
    try:
        sess.set_workers(w0, w1)
        sess.rounds(int(budget["rounds"]))
        rep = sess.report()
        L_sum, L_len = global_L(rep["L_sum"], rep["accepts"], group, comm_device)
        s_lo, s_hi = size_range(policy, m)
        s_opt = s_opt_from(L_sum, L_len, s_lo, s_hi)
        f_local = sess.recheck(s_opt)
        f_best, w_best = pick_best(f_local, w0, group, comm_device)
        owner = next(r for r in range(world) if worker_range(W, r, world)[0] <= w_best < worker_range(W, r, world)[1])
        C = sess.worker_centroids(w_best) if owner == rank else None
        C = broadcast_centroids(C, owner, (k, Xd.shape[1]), group, comm_device).to(Xd.device)
    finally:
        sess.close()
    Y, f_full, _ = native.assign(Xd, C, stream=stream)
    return C, Y, dict(s_opt=s_opt, best_worker=w_best, f_full=f_full, L_sum=L_sum, L_len=L_len,
                      workers=(w0, w1), f_recheck_best=f_best)
