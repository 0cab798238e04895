"""GPU tests of bigmeans_fit_dt: the storage type of X and the mode of the
full-data pass, through the fit entry point.

* BM_F32 with BM_MODE_EXACT is bigmeans_fit: the same C, labels and f, and
  the labels and f(C, X) of the CPU oracle's exact mode for that C (Eq. 1);
* BM_MODE_FAST runs the same fit (the same C), then takes the labels and f
  from the precision pass (tau = 1e-3): they equal bm_assign_bf16 on the
  packed rows with that C, whether X is given in FP32 (packed inside) or
  packed by the caller (BM_BF16 with its FP32 master); the labels equal the
  oracle's except at near ties, and f is within the precision form's error;
* an unknown dt or mode, or BM_BF16 without its master, is BM_EINVAL.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import kmeans as okm  # noqa: E402
from paper_2403_18766_gb300 import native  # noqa: E402
from paper_2403_18766_gb300.synthetic import gaussian_mixture  # noqa: E402

K = 8


def _setup(n=16, m=20_000, seed=41):
    X = gaussian_mixture(m, n, K, seed=seed)
    pol = native.make_policy(s_min=500, s_max=4000, workers=4, passes=3)
    bud = native.make_budget(rounds=2)
    return X, torch.from_numpy(X).cuda(), pol, bud


@pytest.mark.parametrize("n", [16, 40])
def test_exact_mode_is_bigmeans_fit(n):
    X, Xd, pol, bud = _setup(n=n)
    C0, Y0, r0 = native.fit(Xd, K, pol, bud, seed=5)
    C1, Y1, r1 = native.fit_dt(Xd, K, pol, bud, seed=5, mode=native.BM_MODE_EXACT)
    assert torch.equal(C0, C1) and torch.equal(Y0, Y1) and r0["f_full"] == r1["f_full"]
    lab, dist = okm.assign(X, C1.cpu().numpy())
    assert np.array_equal(Y1.cpu().numpy(), lab) and r1["f_full"] == okm.exact_sum(dist)


@pytest.mark.parametrize("n", [16, 40])
def test_fast_mode_takes_the_precision_pass(n):
    X, Xd, pol, bud = _setup(n=n, seed=43)
    C0, Y0, r0 = native.fit_dt(Xd, K, pol, bud, seed=9, mode=native.BM_MODE_EXACT)
    C1, Y1, r1 = native.fit_dt(Xd, K, pol, bud, seed=9, mode=native.BM_MODE_FAST)
    assert torch.equal(C0, C1)                                   # the same fit
    P = native.PackedBF16(Xd)
    Yb, fb, rb = native.assign_bf16(P, C1, tau=1e-3)
    assert torch.equal(Y1, Yb) and r1["f_full"] == fb and r1["rescored_rows"] == rb["rescored_rows"]
    C2, Y2, r2 = native.fit_dt(P, K, pol, bud, seed=9, mode=native.BM_MODE_FAST)   # caller-packed
    assert torch.equal(C2, C1) and torch.equal(Y2, Y1) and r2["f_full"] == r1["f_full"]
    lab, dist = okm.assign(X, C1.cpu().numpy())
    mism = int((Y1.cpu().numpy() != lab).sum())
    assert mism <= max(3, X.shape[0] // 1000)
    fo = okm.exact_sum(dist)
    assert abs(r1["f_full"] - fo) <= 5e-3 * fo


def test_invalid_dtype_mode_and_master():
    _, Xd, pol, bud = _setup()
    m, n = Xd.shape
    C = torch.empty((K, n), dtype=torch.float32, device="cuda")
    rep = native.Report()

    def call(dt, mode, master):
        return native.lib.bigmeans_fit_dt(native._ptr(Xd), native._ptr(master), dt, m, n, K, ctypes.byref(pol),
                                          ctypes.byref(bud), 1, mode, native._stream(None), native._ptr(C),
                                          native._ptr(None), ctypes.byref(rep))

    assert call(7, native.BM_MODE_EXACT, None) == native.BM_EINVAL
    assert call(native.BM_F32, 5, None) == native.BM_EINVAL
    assert call(native.BM_BF16, native.BM_MODE_FAST, None) == native.BM_EINVAL        # no master
    other = Xd.clone()
    assert call(native.BM_F32, native.BM_MODE_EXACT, other) == native.BM_EINVAL       # master not X
    assert call(native.BM_F32, native.BM_MODE_EXACT, Xd) == native.BM_OK              # master = X is fine
    C300 = torch.empty((300, n), dtype=torch.float32, device="cuda")
    st = native.lib.bigmeans_fit_dt(native._ptr(Xd), native._ptr(None), native.BM_F32, m, n, 300,
                                    ctypes.byref(native.make_policy(s_min=600, s_max=4000, workers=2, passes=1)),
                                    ctypes.byref(bud), 1, native.BM_MODE_FAST, native._stream(None), native._ptr(C300),
                                    native._ptr(None), ctypes.byref(rep))
    assert st == native.BM_EINVAL and "k <= 256" in native.lib.bm_last_error().decode()
