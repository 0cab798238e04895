"""GPU tests of the serving context (continuous batching).

* every job's result (C bits, labels, f) is the same alone and in a mix of
  concurrently running jobs, the same as bigmeans_fit_host, and the same as
  the CPU oracle's Algorithm 1 on that job;
* admission keeps the device memory in use under the budget, runs jobs
  concurrently when they fit, and queues them when they do not;
* a small job may overtake a large one that does not fit yet (first fit).
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import bigmeans as obm  # noqa: E402
from paper_2403_18766_gb300 import native  # noqa: E402
from paper_2403_18766_gb300.synthetic import gaussian_mixture  # noqa: E402

JOBS = [  # (m, n, k, s_min, s_max, workers, passes, rounds, seed)
    (60_000, 8, 5, 500, 4000, 4, 3, 2, 1),
    (120_000, 16, 25, 1000, 12_000, 8, 2, 2, 2),
    (30_000, 32, 10, 300, 3000, 4, 2, 3, 3),
    (200_000, 4, 10, 2000, 20_000, 6, 2, 2, 4),
    (80_000, 16, 50, 1000, 8000, 4, 2, 2, 5),
    (45_000, 64, 8, 400, 5000, 3, 2, 2, 6),
]


def _spec(j):
    m, n, k, lo, hi, W, p, T, seed = j
    X = torch.from_numpy(gaussian_mixture(m, n, max(2, k // 2), seed=100 + seed)).pin_memory()
    return X, k, native.make_policy(s_min=lo, s_max=hi, workers=W, passes=p), native.make_budget(rounds=T), seed


def _same(a, b):
    assert a["status"] == native.BM_OK and b["status"] == native.BM_OK
    assert torch.equal(a["C"].view(torch.int32), b["C"].view(torch.int32))
    assert torch.equal(a["labels"], b["labels"])
    assert a["f_full"] == b["f_full"] and a["s_opt"] == b["s_opt"]


def test_results_alone_equal_results_in_the_mix():
    specs = [_spec(j) for j in JOBS]
    ctx = native.ServeContext(64 << 30, 4)
    alone = []
    for X, k, pol, bud, seed in specs:                 # one at a time
        jid = ctx.submit(X, k, pol, bud, seed)
        alone.append(ctx.wait(jid))
    ids = [ctx.submit(X, k, pol, bud, seed) for X, k, pol, bud, seed in specs]   # all at once
    mixed = [ctx.wait(j) for j in ids]
    st = ctx.stats()
    ctx.close()
    for a, b in zip(alone, mixed):
        _same(a, b)
    assert st["peak_active"] >= 2                      # jobs did overlap on the device
    # jobs taken from the mix against the CPU oracle (Algorithm 1, exact mode)
    for i in (0, 5):
        m, n, k, lo, hi, W, p, T, seed = JOBS[i]
        ref = obm.bigmeans(specs[i][0].numpy(), k, dict(s_min=lo, s_max=hi, workers=W, passes=p),
                           dict(rounds=T, max_lloyd=300, tol=1e-4, kpp_candidates=3), seed)
        assert np.array_equal(mixed[i]["C"].numpy().view(np.int32), ref["C"].view(np.int32))
        assert np.array_equal(mixed[i]["labels"].numpy(), ref["labels"])
        assert mixed[i]["f_full"] == ref["f_full"] and mixed[i]["s_opt"] == ref["s_opt"]
    # and the same as the plain host-buffer fit
    X, k, pol, bud, seed = specs[1]
    C, Y, rep = native.fit_host(X, k, pol, bud, seed=seed)
    assert np.array_equal(C.view(np.int32), alone[1]["C"].numpy().view(np.int32))
    assert np.array_equal(Y, alone[1]["labels"].numpy()) and rep["f_full"] == alone[1]["f_full"]


def test_admission_respects_the_budget():
    specs = [_spec(j) for j in JOBS]
    probe = native.ServeContext(64 << 30, 1)
    fps = []
    for X, k, pol, bud, seed in specs:
        jid = probe.submit(X, k, pol, bud, seed)
        fps.append(probe.wait(jid)["footprint_bytes"])
    probe.close()
    budget = int(sorted(fps)[-1] + sorted(fps)[-2] * 0.5)   # about two jobs at a time
    ctx = native.ServeContext(budget, 6)
    ids = [ctx.submit(X, k, pol, bud, seed) for X, k, pol, bud, seed in specs]
    res = [ctx.wait(j) for j in ids]
    st = ctx.stats()
    ctx.close()
    assert all(r["status"] == native.BM_OK for r in res)
    assert st["peak_in_use_bytes"] <= budget
    assert 1 <= st["peak_active"] < 6                   # some jobs had to queue
    assert st["in_use_bytes"] == 0 and st["done"] == len(JOBS)
    # at every job's admission, the jobs running then fit the budget together
    for r in res:
        running = [q for q in res if q["t_admit_s"] <= r["t_admit_s"] < q["t_done_s"]]
        assert sum(q["footprint_bytes"] for q in running) <= budget


def test_small_job_overtakes_a_large_one_that_does_not_fit():
    big = _spec((400_000, 16, 25, 2000, 40_000, 8, 2, 2, 7))
    small = _spec((20_000, 8, 5, 500, 2000, 2, 2, 1, 8))
    first = _spec((300_000, 16, 25, 2000, 30_000, 8, 5, 8, 9))       # long enough to be running
    probe = native.ServeContext(64 << 30, 1)
    fp = {}
    for name, (X, k, pol, bud, seed) in [("big", big), ("small", small), ("first", first)]:
        fp[name] = probe.wait(probe.submit(X, k, pol, bud, seed))["footprint_bytes"]
    probe.close()
    budget = fp["first"] + fp["small"] + (fp["big"] - 1 - fp["small"]) // 2
    assert fp["first"] + fp["big"] > budget >= fp["first"] + fp["small"]
    ctx = native.ServeContext(budget, 4)
    i_first = ctx.submit(*first[:4], seed=first[4])
    time.sleep(0.005)
    i_big = ctx.submit(*big[:4], seed=big[4])
    i_small = ctx.submit(*small[:4], seed=small[4])
    r_first, r_big, r_small = ctx.wait(i_first), ctx.wait(i_big), ctx.wait(i_small)
    ctx.close()
    assert r_big["t_admit_s"] > r_first["t_admit_s"] and r_big["t_submit_s"] < r_first["t_done_s"]
    assert r_small["t_admit_s"] < r_big["t_admit_s"]      # overtook the large job
    assert r_big["t_admit_s"] >= r_first["t_done_s"] - 1e-3 or r_big["t_admit_s"] >= r_small["t_done_s"] - 1e-3


def test_poll_reports_queued_and_running_states():
    X, k, pol, bud, seed = _spec((150_000, 16, 25, 2000, 15_000, 8, 3, 2, 10))
    ctx = native.ServeContext(64 << 30, 1)
    a = ctx.submit(X, k, pol, bud, seed)
    b = ctx.submit(X, k, pol, bud, seed + 1)
    pb = ctx.poll(b)
    assert pb["status"] == native.BM_EAGAIN and pb["state"] in (0, 1)
    ra, rb = ctx.wait(a), ctx.wait(b)
    ctx.close()
    assert ra["state"] == rb["state"] == 2 and rb["t_admit_s"] >= ra["t_done_s"] - 1e-3


def test_many_concurrent_jobs_of_different_shapes():
    """24 jobs with six different (n, k) at once, six running together: every
    job succeeds and equals its result alone (kernels of different shapes
    launched from several host threads share no launch state)."""
    specs = [_spec(JOBS[i % len(JOBS)][:8] + (20 + i,)) for i in range(24)]
    ctx = native.ServeContext(64 << 30, 6)
    ids = [ctx.submit(X, k, pol, bud, seed) for X, k, pol, bud, seed in specs]
    mixed = [ctx.wait(j) for j in ids]
    st = ctx.stats()
    for r in mixed:
        assert r["status"] == native.BM_OK, r.get("error")
    assert st["peak_active"] >= 3
    for i in (0, 7, 17):
        X, k, pol, bud, seed = specs[i]
        _same(ctx.wait(ctx.submit(X, k, pol, bud, seed)), mixed[i])
    ctx.close()


def test_bf16_stored_job_takes_labels_and_f_from_the_precision_pass():
    """A job with BF16 storage fits on the FP32 master (same centroids as the
    FP32 job), then takes its labels and f(C, X) from the BF16 tensor-core
    pass over its packed copy."""
    X, k, pol, bud, seed = _spec(JOBS[1])
    ctx = native.ServeContext(64 << 30, 2)
    rb = ctx.wait(ctx.submit(X, k, pol, bud, seed, bf16=True, tau=1e-3))
    r32 = ctx.wait(ctx.submit(X, k, pol, bud, seed))
    st = ctx.stats()
    ctx.close()
    assert rb["status"] == native.BM_OK, rb.get("error")
    assert torch.equal(rb["C"].view(torch.int32), r32["C"].view(torch.int32))
    assert rb["report"]["f_full"] == r32["f_full"]            # exact objective of the same C
    Xd = X.cuda()
    Y, f, _ = native.assign_bf16(native.PackedBF16(Xd), rb["C"].cuda(), tau=1e-3)
    assert torch.equal(rb["labels"], Y.cpu()) and rb["f_full"] == f
    assert abs(rb["f_full"] - r32["f_full"]) <= 1e-3 * r32["f_full"]
    assert st["in_use_bytes"] == 0
