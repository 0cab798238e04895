"""Failure detection without a GPU fault.

* A bounded device wait that runs out: the test shortens the limit of the
  tensor-core exact pass's mbarrier waits (bm_debug_set_wait_limit) so far
  that the first wait for a tile's copy gives up.  The kernel stops every
  role, waits for its copies and MMAs in flight, frees its tensor memory and
  returns; the call reports BM_ETIMEOUT, and the next call on the same stream
  with the default limit returns the oracle's labels and f(C, X) bit for bit.
* A device allocation that fails (bm_debug_fail_allocs): the fit returns
  BM_ENOMEM and releases what it had taken; in a serving context the job is
  reported done with BM_ENOMEM, no memory stays accounted as in use, and the
  next job runs normally.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import kmeans as okm  # noqa: E402
from paper_2403_18766_gb300 import native  # noqa: E402
from paper_2403_18766_gb300.synthetic import gaussian_mixture  # noqa: E402


@pytest.fixture
def tensor_pass():
    native.set_fullpass_impl(2)
    yield
    native.debug_set_wait_limit(0)
    native.set_fullpass_impl(0)


def test_wait_that_runs_out_reports_timeout_and_the_next_call_is_exact(tensor_pass):
    X = gaussian_mixture(8192, 16, 12, seed=61)
    C = X[np.random.default_rng(61).integers(0, X.shape[0], 25)].copy()
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()
    lab, dist = okm.assign(X, C)
    f_ref = okm.exact_sum(dist)
    native.debug_set_wait_limit(1, 0)              # one plain poll per wait
    timeouts = 0
    for _ in range(4):
        try:
            Y, f, _ = native.assign(Xd, Cd)
        except native.BigmeansError as e:
            assert e.status == native.BM_ETIMEOUT, str(e)
            timeouts += 1
            continue
        assert native.last_fullpass_impl() == 2
        assert np.array_equal(Y.cpu().numpy(), lab) and f == f_ref   # a call that did not run out
    assert timeouts >= 1
    native.debug_set_wait_limit(0)                 # default limit
    for _ in range(2):
        Y, f, rep = native.assign(Xd, Cd)
        assert native.last_fullpass_impl() == 2
        assert np.array_equal(Y.cpu().numpy(), lab) and f == f_ref


def test_failed_allocation_in_a_fit_is_enomem_and_leaves_nothing_behind():
    X = torch.from_numpy(gaussian_mixture(20_000, 8, 5, seed=62)).cuda()
    pol = native.make_policy(s_min=500, s_max=4000, workers=3, passes=2)
    bud = native.make_budget(rounds=2)
    C0, Y0, r0 = native.fit(X, 5, pol, bud, seed=4)
    native.debug_fail_allocs(1)
    try:
        with pytest.raises(native.BigmeansError) as e:
            native.fit(X, 5, pol, bud, seed=4)
        assert e.value.status == native.BM_ENOMEM
    finally:
        native.debug_fail_allocs(0)
    C1, Y1, r1 = native.fit(X, 5, pol, bud, seed=4)
    assert torch.equal(C0.view(torch.int32), C1.view(torch.int32)) and torch.equal(Y0, Y1)
    assert r0["f_full"] == r1["f_full"]


def test_failed_allocation_of_a_served_job_keeps_the_context_serving():
    X = torch.from_numpy(gaussian_mixture(30_000, 8, 5, seed=63)).pin_memory()
    pol = native.make_policy(s_min=500, s_max=4000, workers=3, passes=2)
    bud = native.make_budget(rounds=2)
    ctx = native.ServeContext(8 << 30, 1)
    native.debug_fail_allocs(1)
    try:
        bad = ctx.wait(ctx.submit(X, 5, pol, bud, seed=6))
    finally:
        native.debug_fail_allocs(0)
    assert bad["state"] == 2 and bad["status"] == native.BM_ENOMEM, bad
    assert bad["error"]
    st = ctx.stats()
    assert st["in_use_bytes"] == 0 and st["active"] == 0
    good = ctx.wait(ctx.submit(X, 5, pol, bud, seed=6))
    ctx.close()
    C, Y, rep = native.fit_host(X, 5, pol, bud, seed=6)
    assert good["status"] == native.BM_OK
    assert np.array_equal(good["C"].numpy().view(np.int32), C.view(np.int32))
    assert np.array_equal(good["labels"].numpy(), Y) and good["f_full"] == rep["f_full"]
