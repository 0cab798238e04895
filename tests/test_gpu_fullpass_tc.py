"""GPU parity of the tensor-core exact full pass (tcgen05 kind::tf32 proposal,
certified, uncertain rows re-scored in the FP32 direct form).

Labels and f(C, X) must equal the oracle bit for bit, and equal those of the
FP32-ALU pass, for every shape the tensor-core pass takes (n % 4 == 0): one and
two 32-float column blocks, k up to 256, tiles with ragged tails, m below one
tile, ties between duplicated centroids and data far from the origin (where
the TF32 error bound makes many rows uncertain).  Ineligible inputs (n % 4 !=
0) must fall back to the FP32-ALU pass with the same results.
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


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(autouse=True)
def _default_impl():
    native.set_fullpass_impl(0)
    yield
    native.set_fullpass_impl(0)


def _both(X, C):
    """(tensor-core pass where it applies, FP32-ALU pass) on the same input."""
    Xd, Cd = _t(X), _t(C)
    native.set_fullpass_impl(2)
    Y0, f0, r0 = native.assign(Xd, Cd)
    impl0 = native.last_fullpass_impl()
    native.set_fullpass_impl(1)
    Y1, f1, r1 = native.assign(Xd, Cd)
    impl1 = native.last_fullpass_impl()
    native.set_fullpass_impl(0)
    return (Y0.cpu().numpy(), f0, r0, impl0), (Y1.cpu().numpy(), f1, r1, impl1)


SHAPES = [(1, 4, 1), (127, 4, 3), (128, 8, 5), (4097, 16, 25), (100_003, 16, 25), (30_001, 64, 100),
          (20_000, 32, 50), (9_999, 36, 17), (50_000, 32, 256), (70_001, 12, 9), (3000, 20, 200),
          (257, 64, 1)]


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_tensor_core_pass_is_bit_exact(m, n, k):
    X = gaussian_mixture(m, n, max(1, k // 2), seed=3 * m + k)
    C = X[np.random.default_rng(k + 1).integers(0, m, k)].copy()
    (Y0, f0, r0, i0), (Y1, f1, r1, i1) = _both(X, C)
    assert (i0, i1) == (2, 1)
    lab, dist = okm.assign(X, C)
    assert np.array_equal(Y0, lab)
    assert f0 == okm.exact_sum(dist)
    assert np.array_equal(Y1, Y0) and f1 == f0
    assert r0["inexact_terms"] == 0


def test_widest_case_both_passes():
    """n = 64, k = 176: the widest shape the tensor-core pass takes (its
    B operands and stages fill the shared memory)."""
    X = gaussian_mixture(20_000, 64, 88, seed=21)
    C = X[np.random.default_rng(3).integers(0, X.shape[0], 176)].copy()
    (Y0, f0, _, i0), (Y1, f1, _, i1) = _both(X, C)
    assert (i0, i1) == (2, 1)
    lab, dist = okm.assign(X, C)
    assert np.array_equal(Y0, lab) and f0 == okm.exact_sum(dist)
    assert np.array_equal(Y1, Y0) and f1 == f0


@pytest.mark.parametrize("n,k,want", [(16, 25, 1), (16, 50, 2), (32, 10, 1), (32, 50, 2), (64, 25, 1), (64, 100, 2),
                                     (3, 100, 1)])
def test_default_choice_by_shape(n, k, want):
    """impl 0 takes the tensor cores once n_pad * k > 512 (n_pad <= 32) or
    > 1600 (n_pad = 64), where n % 4 == 0."""
    X = gaussian_mixture(5000, n, 6, seed=n + k)
    C = X[np.random.default_rng(k).integers(0, X.shape[0], k)].copy()
    native.set_fullpass_impl(0)
    Y, f, _ = native.assign(_t(X), _t(C))
    assert native.last_fullpass_impl() == want
    lab, dist = okm.assign(X, C)
    assert np.array_equal(Y.cpu().numpy(), lab) and f == okm.exact_sum(dist)


def test_ties_between_duplicated_centroids():
    X = np.float32([[0, 0, 1, 1], [1, 1, 0, 0], [5, 5, 5, 5], [2, 2, 2, 2]] * 700)
    C = np.float32([[1, 1, 0, 0], [0, 0, 1, 1], [1, 1, 0, 0], [5, 5, 5, 5], [2, 2, 2, 2], [2, 2, 2, 2]])
    (Y0, f0, r0, i0), (Y1, f1, _, _) = _both(X, C)
    assert i0 == 2
    lab, dist = okm.assign(X, C)
    assert np.array_equal(Y0, lab) and f0 == okm.exact_sum(dist)
    assert r0["rescored_rows"] >= 1400              # half of the rows tie with a duplicate
    assert np.array_equal(Y1, Y0) and f1 == f0


def test_far_from_origin_many_uncertain_rows():
    X = gaussian_mixture(40_000, 16, 8, seed=5) + np.float32(3000.0)
    C = X[np.random.default_rng(2).integers(0, X.shape[0], 12)].copy()
    (Y0, f0, r0, i0), (Y1, f1, _, _) = _both(X, C)
    assert i0 == 2
    lab, dist = okm.assign(X, C)
    assert np.array_equal(Y0, lab) and f0 == okm.exact_sum(dist)
    assert r0["rescored_rows"] > 1000
    assert np.array_equal(Y1, Y0) and f1 == f0


@pytest.mark.parametrize("n", [2, 3, 17, 33])
def test_ineligible_widths_fall_back(n):
    X = gaussian_mixture(5000, n, 4, seed=n)
    C = X[:7].copy()
    (Y0, f0, _, i0), (Y1, f1, _, i1) = _both(X, C)
    assert (i0, i1) == (1, 1)
    lab, dist = okm.assign(X, C)
    assert np.array_equal(Y0, lab) and f0 == okm.exact_sum(dist)


def test_misaligned_x_is_rejected():
    X = gaussian_mixture(3001, 4, 3, seed=9)
    buf = torch.zeros(3001 * 4 + 1, dtype=torch.float32, device="cuda")
    buf[1:].copy_(torch.from_numpy(X.reshape(-1)))
    Xd = buf[1:].view(3001, 4)                       # 4-byte aligned only
    with pytest.raises(native.BigmeansError, match="aligned"):
        native.assign(Xd, _t(X[:5].copy()))


def test_bad_impl_value_is_rejected():
    with pytest.raises(native.BigmeansError):
        native.set_fullpass_impl(7)
    with pytest.raises(native.BigmeansError):
        native.set_fullpass_impl(-1)
