"""bm_assign_noalloc against bm_assign, through the C ABI.

bm_assign_noalloc serves callers that cannot allocate device memory when
they need a full-data assignment (for instance services that keep all of
their device memory in their own pool).  It keeps its scratch in a fixed
array inside the library, so two calls in a row must each start from cleared
accumulators and reproduce bm_assign exactly.  This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2403_18766_gb300 import native  # noqa: E402
from paper_2403_18766_gb300.synthetic import gaussian_mixture  # noqa: E402


def _case(m, n, k, seed):
    X = gaussian_mixture(m, n, max(2, k // 2), seed=seed)
    C = X[np.random.default_rng(seed).integers(0, m, k)].copy()
    return torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()


@pytest.fixture(params=[0, 2], ids=["impl-by-shape", "impl-tensor-cores"])
def fullpass_impl(request):
    native.set_fullpass_impl(request.param)
    yield request.param
    native.set_fullpass_impl(0)


def test_noalloc_matches_bm_assign_two_calls_in_a_row(fullpass_impl):
    """By shape: n = 16, k = 25 and n = 33 take the FP32-ALU pass, n = 64,
    k = 100 the tensor-core pass; with impl 2 every case with n % 4 == 0
    takes the tensor-core pass through the same fixed scratch."""
    cases = [_case(100_003, 16, 25, 1), _case(40_000, 33, 40, 2), _case(60_001, 64, 100, 3)]
    expect_tc = {0: [False, False, True], 2: [True, False, True]}[fullpass_impl]
    for _ in range(2):                          # the scratch keeps the previous call's contents
        for (X, C), tc in zip(cases, expect_tc):
            Y_ref, f_ref, _ = native.assign(X, C)
            Y, f = native.assign_noalloc(X, C)
            torch.cuda.synchronize()
            assert native.last_fullpass_impl() == (2 if tc else 1)
            assert torch.equal(Y, Y_ref)
            assert f == f_ref                  # exact objective: bit-identical doubles


def test_noalloc_rejects_sizes_above_its_scratch():
    X, _ = _case(1000, 64, 2, 3)
    C = X[:300].clone()                        # 300 * 64 floats > 16,384
    with pytest.raises(native.BigmeansError) as e:
        native.assign_noalloc(X, C)
    assert e.value.status == native.BM_EINVAL
    assert "scratch" in str(e.value)
