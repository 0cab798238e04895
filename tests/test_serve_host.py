"""Host-side checks of the serving context (no GPU needed): argument checks,
admission bound (a job larger than the whole budget is refused at submit),
and the footprint the admission uses."""
import numpy as np
import pytest

from paper_2403_18766_gb300 import native


def _pol(workers=4, passes=2, s_max=5000):
    return native.make_policy(s_min=1000, s_max=s_max, workers=workers, passes=passes)


def test_create_checks_arguments():
    for budget, active in [(0, 2), (-5, 2), (1 << 30, 0), (1 << 30, 65)]:
        with pytest.raises(native.BigmeansError):
            native.ServeContext(budget, active)
    ctx = native.ServeContext(1 << 30, 3)
    st = ctx.stats()
    assert st["budget_bytes"] == 1 << 30 and st["active"] == 0 and st["queued"] == 0 and st["done"] == 0
    ctx.close()


def test_submit_refuses_jobs_above_the_budget_and_bad_shapes():
    ctx = native.ServeContext(1 << 20, 2)                 # 1 MB: no fit fits
    X = np.zeros((100_000, 16), np.float32)
    with pytest.raises(native.BigmeansError) as e:
        ctx.submit(X, 25, _pol(), native.make_budget(rounds=1))
    assert e.value.status == native.BM_ENOMEM
    with pytest.raises(native.BigmeansError) as e:
        ctx.submit(np.zeros((100, 80), np.float32), 5, _pol(s_max=100), native.make_budget(rounds=1))
    assert e.value.status == native.BM_EINVAL
    with pytest.raises(native.BigmeansError) as e:          # s_min below k
        ctx.submit(np.zeros((5000, 4), np.float32), 2000, _pol(), native.make_budget(rounds=1))
    assert e.value.status == native.BM_EINVAL
    assert ctx.stats()["queued"] == 0
    ctx.close()


def test_footprint_is_workspace_plus_buffers():
    pol, bud = _pol(workers=8), native.make_budget(rounds=2)
    m, n, k = 200_000, 16, 25
    ws = native.fit_footprint(m, n, k, pol, bud)
    job = native.Job(X_host=1, m=m, n=n, k=k, policy=pol, budget=bud, seed=0, C_out_host=1, labels_out_host=1)
    fp = __import__("ctypes").c_int64(0)
    assert native.lib.bm_job_footprint(__import__("ctypes").byref(job), __import__("ctypes").byref(fp)) == 0
    assert fp.value >= ws + m * n * 4 + k * n * 4 + m * 4
    assert fp.value - (ws + m * n * 4 + k * n * 4 + m * 4) < 4096
    # more workers or larger samples need more workspace; m alone only changes the tables
    assert native.fit_footprint(m, n, k, _pol(workers=16), bud) > ws
    assert native.fit_footprint(m, n, k, _pol(workers=8, s_max=50_000), bud) > ws


def test_cluster_tile_setting_is_checked():
    assert native.get_rows_per_cta() == 1024
    for bad in (-1, 100, 40_000):
        with pytest.raises(native.BigmeansError):
            native.set_rows_per_cta(bad)
    native.set_rows_per_cta(4096)
    assert native.get_rows_per_cta() == 4096
    native.set_rows_per_cta(0)
    assert native.get_rows_per_cta() == 1024
