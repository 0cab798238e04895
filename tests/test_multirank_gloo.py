"""The N > 1 path of bench.py on CPU: two gloo ranks.  The ranks run one fit
together (each its own workers, weak scaling, the same seed); the whole-job
time is the slowest rank's and the work is the sum over ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_local = 1.0 + 0.5 * rank                     # rank 1 is the slow one
        work_local = 100.0 * (rank + 1)
        t, w = bench.aggregate(t_local, work_local, "cpu")
        out.put((rank, t, w, bench.rank_seed(rank), bench._dist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_total_work():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, w, seed, (ws, rk) in res:
        assert t == 1.5 and w == 300.0                  # max over ranks, sum over ranks
        assert ws == 2 and rk == rank
    assert res[0][3] == res[1][3]                       # one fit: the same seed on every rank
