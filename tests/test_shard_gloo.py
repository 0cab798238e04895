"""The exchange of a fit sharded over ranks, on CPU: two gloo ranks.

Each rank takes the recorded results of its workers from one oracle run of
Algorithm 1 (workload 1: 10^4 x 2, k = 5, 4 workers, T = 2 rounds, p = 10):
the sizes it added to L and, on the common sample, each worker's f_hat and
centroids.  The ranks then exchange through paper_2403_18766_gb300.shard
(an all-gather of (sum of L, |L|), an all-gather of the least (f_hat, w), a
broadcast of the winner's centroids) and must arrive at the single-process
oracle's s_opt, best worker and C_best.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
POLICY = dict(set=[250, 500, 1000, 2000], workers=4, passes=10)
BUDGET = dict(rounds=2, max_lloyd=300, tol=1e-4, kpp_candidates=3)
SEED = 2024


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle():
    from oracle import bigmeans as obm
    from paper_2403_18766_gb300.synthetic import workload
    X = workload("gmm_10k_n2_k5")
    return X, obm.bigmeans(X, 5, POLICY, BUDGET, SEED)


def _worker_L(ref, w):
    """Sizes worker w added to L, from the oracle's log (one entry per accepted pass)."""
    P = POLICY["passes"]
    acc = ref["log"]["accepts"][w]
    return [ref["log"]["sizes"][w][i // P] for i, a in enumerate(acc) if a]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    from paper_2403_18766_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, ref = _oracle()
        W = POLICY["workers"]
        w0, w1 = shard.worker_range(W, rank, world)
        L = [s for w in range(w0, w1) for s in _worker_L(ref, w)]
        L_sum, L_len = shard.global_L(sum(L), len(L), None, "cpu")
        s_lo, s_hi = shard.size_range(POLICY, X.shape[0])
        s_opt = shard.s_opt_from(L_sum, L_len, s_lo, s_hi)
        f_local = [ref["f_hat"][w] for w in range(w0, w1)]
        f_best, w_best = shard.pick_best(f_local, w0, None, "cpu")
        owner = next(r for r in range(world) if shard.worker_range(W, r, world)[0] <= w_best
                     < shard.worker_range(W, r, world)[1])
        C = ref["C_workers"][w_best] if owner == rank else None
        C = shard.broadcast_centroids(C, owner, (5, X.shape[1]), None, "cpu").numpy()
        out.put((rank, s_opt, w_best, f_best, C.tobytes(), L_len, (w0, w1)))
    finally:
        dist.destroy_process_group()


def test_sharded_exchange_equals_the_single_process_oracle():
    sys.path.insert(0, ROOT)
    X, ref = _oracle()
    assert sum(len(_worker_L(ref, w)) for w in range(POLICY["workers"])) == len(ref["L"])
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][6] == (0, 2) and res[1][6] == (2, 4)
    for rank, s_opt, w_best, f_best, C, L_len, _ in res:
        assert s_opt == ref["s_opt"]
        assert w_best == ref["best_worker"]
        assert f_best == ref["f_hat"][ref["best_worker"]]
        assert C == np.ascontiguousarray(ref["C"], dtype=np.float32).tobytes()
        assert L_len == len(ref["L"])


def test_size_range_and_mean_rule():
    sys.path.insert(0, ROOT)
    from paper_2403_18766_gb300 import shard
    assert shard.size_range(dict(s_min=100, s_max=10**9), 5000) == (100, 5000)
    assert shard.size_range(dict(set=[30, 9000, 700]), 5000) == (30, 5000)
    assert shard.s_opt_from(0, 0, 10, 99) == 99                 # empty L: s_max
    assert shard.s_opt_from(5, 2, 1, 99) == 3                   # 2.5 rounds half up
    assert shard.s_opt_from(400, 2, 1, 99) == 99                # clipped
    assert shard.worker_range(16, 1, 3) == (5, 10)
