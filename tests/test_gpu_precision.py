"""GPU tests of the precision form: BF16 pack and the tensor-core full pass.

* the packed rows are torch's round-to-nearest bfloat16 of X, in the
  documented swizzled layout, and the norms are fl(sum bf16(x)^2);
* tau = inf re-scores every row with the exact FP32 definition, so labels and
  f equal bm_assign and the CPU oracle bit for bit (checks the bookkeeping of
  the kernel);
* tau = 0 takes every label from the tensor cores: they must equal the argmin
  of a bfloat16 / FP32-accumulate reference except where two centroids are
  within the accumulation error (checks descriptors, swizzle, TMEM reads);
* the default tau = 1e-3 agrees with the exact pass on all but near ties and
  reports how far its objective is from the exact one;
* the certified variant's labels equal the oracle's exact-mode labels.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import kmeans as okm  # noqa: E402
from paper_2403_18766_gb300 import native  # noqa: E402
from paper_2403_18766_gb300.synthetic import gaussian_mixture  # noqa: E402


def _case(m, n, k, seed, components=None):
    X = gaussian_mixture(m, n, components or max(2, k // 2), seed=seed)
    C = X[np.random.default_rng(seed).integers(0, m, k)].copy()
    return torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()


_ORACLE = {}


def _oracle(X, C, key):
    """Exact-mode labels and f(C, X) from the CPU oracle (Eq. 1), cached per case."""
    if key not in _ORACLE:
        lab, dist = okm.assign(X.cpu().numpy(), C.cpu().numpy())
        _ORACLE[key] = (lab, okm.exact_sum(dist))
    return _ORACLE[key]


def _unswizzle(Xb_bytes, m):
    rows = Xb_bytes.view(torch.int16).view(-1, 64).cpu().numpy()
    out = np.empty_like(rows)
    r = np.arange(rows.shape[0])[:, None]
    for c in range(8):
        pc = c ^ (r & 7)
        out[:, 8 * c:8 * c + 8] = np.take_along_axis(rows, (8 * pc + np.arange(8)[None, :]), axis=1)
    return out[:m]


@pytest.mark.parametrize("m,n", [(1000, 64), (333, 17), (129, 8), (5000, 3)])
def test_pack_bf16_layout_and_norms(m, n):
    X, _ = _case(m, n, 2, m + n)
    P = native.PackedBF16(X)
    ref = torch.zeros(m, 64, dtype=torch.bfloat16)
    ref[:, :n] = X.cpu().to(torch.bfloat16)
    got = _unswizzle(P.Xb, m)
    assert np.array_equal(got, ref.view(torch.int16).numpy())
    b = X.cpu().to(torch.bfloat16).float().numpy()
    norms = np.zeros(m, np.float32)
    for d in range(n):                                   # FMA chain in FP32, ascending d
        norms = (norms.astype(np.float64) + b[:, d].astype(np.float64) ** 2).astype(np.float32)
    np.testing.assert_allclose(P.norms[:m].cpu().numpy(), norms, rtol=2e-6, atol=1e-6)
    m_pad = (m + 127) // 128 * 128
    assert torch.all(P.norms[m:m_pad] == 0)
    assert P.norms[m_pad].item() == X.abs().max().item()


# n = 30 (not a multiple of 4): the re-score kernel reads its rows element by
# element; the other n with 16-byte loads
CASES = [(100_003, 64, 100), (5000, 40, 17), (384, 16, 256), (1000, 8, 3), (70_001, 16, 25), (20_011, 30, 40)]


@pytest.mark.parametrize("m,n,k", CASES)
def test_tau_inf_is_the_exact_pass(m, n, k):
    X, C = _case(m, n, k, 7 * m + k)
    P = native.PackedBF16(X)
    Y, f, rep = native.assign_bf16(P, C, tau=math.inf)
    Yr, fr, _ = native.assign(X, C)
    assert torch.equal(Y, Yr)
    assert f == fr
    assert rep["rescored_rows"] == m
    lab, fo = _oracle(X, C, (m, n, k, 7 * m + k))
    assert np.array_equal(Y.cpu().numpy(), lab) and f == fo


@pytest.mark.parametrize("m,n,k", CASES)
def test_tau0_labels_come_from_the_tensor_cores(m, n, k):
    X, C = _case(m, n, k, 11 * m + k)
    P = native.PackedBF16(X)
    Y, f, rep = native.assign_bf16(P, C, tau=0.0)
    assert rep["rescored_rows"] == 0
    xb = X.to(torch.bfloat16).float()
    cb = C.to(torch.bfloat16).float()
    dot = xb.double() @ cb.double().T                    # exact products, FP64 sum
    g = (cb.double() ** 2).sum(1)[None, :] - 2 * dot
    top2 = torch.topk(g, 2, dim=1, largest=False)
    lab = top2.indices[:, 0].int()
    gap = top2.values[:, 1] - top2.values[:, 0]
    scale = (xb.double().abs() @ cb.double().abs().T).max(1).values   # sum |x_d c_d| bound
    clear = gap > 1e-4 * scale + 1e-6                    # far above FP32 accumulation error
    assert clear.float().mean() > 0.5
    assert torch.equal(Y[clear], lab[clear])


@pytest.mark.parametrize("m,n,k", CASES)
def test_default_tau_matches_exact_labels_except_near_ties(m, n, k):
    X, C = _case(m, n, k, 13 * m + k)
    P = native.PackedBF16(X)
    Y, f, rep = native.assign_bf16(P, C, tau=1e-3)
    Yr, fr, _ = native.assign(X, C)
    lab, fo = _oracle(X, C, (m, n, k, 13 * m + k))
    assert np.array_equal(Yr.cpu().numpy(), lab) and fr == fo
    mism = (Y != Yr).nonzero().flatten()
    assert mism.numel() <= max(3, m // 100)
    if mism.numel():
        rows = mism.cpu().numpy()
        Xn, Cn = X.cpu().numpy(), C.cpu().numpy()
        D = okm.d32_all(Xn[rows], Cn)
        srt = np.sort(D, axis=1)
        xx = (Xn[rows].astype(np.float64) ** 2).sum(1)
        assert np.all(srt[:, 1] - srt[:, 0] < 0.05 * xx + 1.0)   # only close calls differ
    assert abs(f - fr) <= 5e-3 * fr


@pytest.mark.parametrize("m,n,k", CASES)
@pytest.mark.parametrize("tau", [0.0, 1e-3])
def test_certified_labels_equal_the_exact_pass(m, n, k, tau):
    """bm_assign_bf16_certified: every label equals bm_assign's (a row keeps
    its tensor-core label only where the BF16 bound proves it), with at least
    the rows of the plain rule re-scored."""
    X, C = _case(m, n, k, 17 * m + k)
    P = native.PackedBF16(X)
    Y, f, rep = native.assign_bf16(P, C, tau=tau, certified=True)
    Yr, fr, _ = native.assign(X, C)
    assert torch.equal(Y, Yr)
    lab, fo = _oracle(X, C, (m, n, k, 17 * m + k))
    assert np.array_equal(Y.cpu().numpy(), lab)
    assert abs(f - fo) <= 5e-3 * fo
    _, _, rep_plain = native.assign_bf16(P, C, tau=tau)
    assert rep["rescored_rows"] >= rep_plain["rescored_rows"]
    assert abs(f - fr) <= 5e-3 * fr


def test_certified_near_ties_and_far_from_origin():
    """Duplicated and nearly duplicated centroids, and data far from the origin
    (where BF16 cannot separate most rows): labels still equal the exact pass."""
    X = gaussian_mixture(20_000, 16, 8, seed=23) + np.float32(500.0)
    C = X[np.random.default_rng(5).integers(0, X.shape[0], 12)].copy()
    C[3] = C[2]
    C[7] = C[6] + np.float32(1e-3)
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()
    P = native.PackedBF16(Xd)
    Y, f, rep = native.assign_bf16(P, Cd, tau=0.0, certified=True)
    Yr, fr, _ = native.assign(Xd, Cd)
    assert torch.equal(Y, Yr)
    lab, _ = okm.assign(X, C)
    assert np.array_equal(Y.cpu().numpy(), lab)
    assert rep["rescored_rows"] > 0


def test_queued_rows_resolved_among_their_candidates():
    """A close call carries the centroids whose BF16 g lies within the
    certificate threshold of the least (at most eight; more are flagged for
    all k).  Groups of 4 and of 11 nearly equal centroids near the origin
    exercise both: with tau = inf every row is queued, and labels and f must
    equal the exact pass and the oracle bit for bit."""
    X = gaussian_mixture(30_000, 32, 6, seed=29)
    rng = np.random.default_rng(31)
    C = X[rng.integers(0, X.shape[0], 20)].copy()
    for j in (1, 2, 3):                                  # 4 centroids within 1e-3 of C[0]
        C[j] = C[0] + np.float32(1e-3 * j)
    for j in range(5, 15):                               # 11 within 1e-2 of C[4]: all k
        C[j] = C[4] - np.float32(1e-3 * (j - 4))
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()
    P = native.PackedBF16(Xd)
    Yr, fr, _ = native.assign(Xd, Cd)
    lab, fo = okm.assign(X, C)
    lab_f = okm.exact_sum(fo)
    assert np.array_equal(Yr.cpu().numpy(), lab) and fr == lab_f
    for certified in (False, True):
        Y, f, rep = native.assign_bf16(P, Cd, tau=math.inf, certified=certified)
        assert rep["rescored_rows"] == X.shape[0]
        assert torch.equal(Y, Yr) and f == fr
    counts = np.bincount(lab, minlength=20)
    assert counts[0:4].sum() > 0 and counts[4:15].sum() > 0   # both groups are nearest to some rows
    Y, f, rep = native.assign_bf16(P, Cd, tau=0.0, certified=True)
    assert torch.equal(Y, Yr)
    assert 0 < rep["rescored_rows"] < X.shape[0]


@pytest.mark.parametrize("tau", [1e-3, math.inf])
def test_rescore_of_aligned_and_misaligned_master_agree(tau):
    """The same FP32 master at a 16-byte aligned and at a misaligned address:
    the re-score kernel reads the queued rows with 16-byte loads in the first
    case and element by element in the second; labels, f and the re-scored
    count agree."""
    m, n, k = 50_021, 32, 60
    X, C = _case(m, n, k, 23)
    P = native.PackedBF16(X)
    Y0, f0, r0 = native.assign_bf16(P, C, tau=tau)
    raw = torch.empty(m * n + 4, dtype=torch.float32, device="cuda")
    Xu = raw[1:1 + m * n].view(m, n)                     # 4 bytes past a 16-byte boundary
    Xu.copy_(X)
    assert Xu.data_ptr() % 16 == 4
    P.X = Xu
    Y1, f1, r1 = native.assign_bf16(P, C, tau=tau)
    assert torch.equal(Y0, Y1) and f0 == f1
    assert r0["rescored_rows"] == r1["rescored_rows"] > 0
    if tau == math.inf:
        assert r0["rescored_rows"] == m
