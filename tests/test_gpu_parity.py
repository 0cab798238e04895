"""GPU parity: every step of the CUDA path against the CPU oracle, through the C ABI.

The bar is bit-exact for everything: indices, gathered rows, labels,
centroids (FP32 bits), iteration counts, empty-cluster flags and objectives
(FP64 bits), because both sides compute the same exactly specified quantities
(FP32 direct-form distances, exact sums rounded once).  Sizes span several
CTA slices and ragged tails; edge cases cover k = 1, s = m, duplicated points,
ties and the largest supported width n = 64.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import bigmeans as obm  # noqa: E402
from oracle import kmeans as okm  # noqa: E402
from oracle import rng as orng  # noqa: E402
from paper_2403_18766_gb300 import native  # noqa: E402
from paper_2403_18766_gb300.synthetic import gaussian_mixture, workload  # noqa: E402

DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _eq_f32(a, b):
    a = np.asarray(a, dtype=np.float32)
    b = np.asarray(b, dtype=np.float32)
    return a.shape == b.shape and np.array_equal(a.view(np.uint32), b.view(np.uint32))


# ------------------------------------------------------------------ a1 sample
@pytest.fixture
def sampler_impl(request):
    native.set_sampler_impl(request.param)
    yield request.param
    native.set_sampler_impl(0)


@pytest.mark.parametrize("sampler_impl", [0, 1], indirect=True)
@pytest.mark.parametrize("m,s", [(1, 1), (7, 0), (50, 50), (1000, 999), (10_000, 2000),
                                 (100_000, 64_000), (1_000_000, 65_537), (3, 2), (257, 256),
                                 (2_500_000, 3000)])
def test_sample_bit_exact(m, s, sampler_impl):
    """Both samplers (shared-memory bitmap where it fits, device tables)
    against the oracle; m = 2.5e6 takes the tables even in the default mode."""
    for purpose, w, t, p in [(orng.P_PASS, 0, 0, 0), (orng.P_EVAL, 3, 7, 0), (orng.P_FINAL, 0, 0, 0)]:
        got = native.sample(12345, purpose, w, t, p, m, s).cpu().numpy()
        ref = obm.sample_indices(12345, purpose, w, t, p, m, s)
        assert np.array_equal(got, ref), (m, s, purpose)


def test_fit_same_with_either_sampler():
    X = gaussian_mixture(60_000, 8, 6, seed=41)
    pol = dict(s_min=2000, s_max=50_000, workers=4, passes=3)
    bud = dict(rounds=2, max_lloyd=300, tol=1e-4, kpp_candidates=3)
    outs = []
    try:
        for impl in (0, 1):
            native.set_sampler_impl(impl)
            outs.append(native.fit(_t(X), 6, native.make_policy(**pol), native.make_budget(**bud), seed=8))
    finally:
        native.set_sampler_impl(0)
    (C0, Y0, r0), (C1, Y1, r1) = outs
    assert torch.equal(C0.view(torch.int32), C1.view(torch.int32)) and torch.equal(Y0, Y1)
    assert r0["f_full"] == r1["f_full"] and r0["s_opt"] == r1["s_opt"]
    ref = obm.bigmeans(X, 6, pol, bud, seed=8)
    _assert_same(C0.cpu().numpy(), Y0.cpu().numpy(), r0, ref)


def test_sampler_impl_value_checked():
    with pytest.raises(native.BigmeansError):
        native.set_sampler_impl(2)
    assert native.get_sampler_impl() == 0


# ------------------------------------------------------------------ a2 gather
@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 33, 64])
def test_gather_bit_exact(n):
    X = gaussian_mixture(5000, n, 3, seed=n)
    idx = obm.sample_indices(9, orng.P_PASS, 0, 0, 0, 5000, 4099)
    S = native.gather(_t(X), _t(idx)).cpu().numpy()
    assert _eq_f32(S, X[idx])


# ---------------------------------------------------------------- a3 kmeans++
@pytest.mark.parametrize("s,n,k,degpat", [(300, 2, 5, "all"), (5000, 2, 5, "all"),
                                          (9001, 16, 25, "all"), (4097, 3, 7, "some"),
                                          (20000, 32, 10, "some"), (3000, 64, 12, "all"),
                                          (500, 5, 1, "all")])
def test_kmeanspp_bit_exact(s, n, k, degpat):
    S = gaussian_mixture(s, n, max(2, k // 2), seed=s + n)
    rs = np.random.default_rng(k)
    if degpat == "all":
        deg = np.ones(k, dtype=bool)
        C0 = np.zeros((k, n), np.float32)
    else:
        deg = rs.random(k) < 0.5
        deg[0] = False
        C0 = S[rs.integers(0, s, k)].copy()
    got = native.kmeanspp(_t(S), _t(C0), deg.astype(np.uint8), 3, 77, 2, 3, 4).cpu().numpy()
    ref, _ = okm.kmeanspp_reseed(S, C0, deg, orng.stream_key(77, orng.P_KPP, 2, 3, 4), 3)
    assert _eq_f32(got, ref)


def test_kmeanspp_duplicates_and_zero_weights():
    S = np.repeat(np.float32([[0, 0], [1, 1], [5, 5]]), 40, axis=0)
    C0 = np.zeros((4, 2), np.float32)
    for trials in (1, 3):
        got = native.kmeanspp(_t(S), _t(C0), np.ones(4, np.uint8), trials, 3, 0, 0, 0).cpu().numpy()
        ref, _ = okm.kmeanspp_reseed(S, C0, np.ones(4, bool), orng.stream_key(3, orng.P_KPP, 0, 0, 0),
                                     trials)
        assert _eq_f32(got, ref)


# ------------------------------------------------------------------ a4-a6 lloyd
@pytest.mark.parametrize("s,n,k,max_iter,tol", [(2000, 2, 5, 300, 1e-4), (4097, 3, 7, 300, 1e-4),
                                                (30001, 16, 25, 300, 1e-4), (12000, 32, 10, 50, 0.0),
                                                (5000, 64, 20, 300, 1e-4), (700, 2, 1, 300, 1e-4),
                                                (999, 4, 6, 0, 1e-4), (4096, 8, 9, 3, -1.0)])
def test_lloyd_bit_exact(s, n, k, max_iter, tol):
    S = gaussian_mixture(s, n, k + 2, seed=s * 7 + k, cov="aniso" if n <= 16 else "iso")
    C0 = S[:: max(1, s // k)][:k].copy()
    C, f, it, empty = native.lloyd(_t(S), _t(C0), max_iter, tol)
    ref = okm.lloyd(S, C0, max_iter, tol)
    assert it == ref["iters"]
    assert _eq_f32(C.cpu().numpy(), ref["C"])
    assert f == ref["f"]
    assert np.array_equal(empty.cpu().numpy(), ref["empty"])


def test_lloyd_empty_cluster_keeps_centroid():
    S = np.float32([[0, 0], [0, 1], [10, 10], [10, 11]] * 50)
    C0 = np.float32([[0, 0.5], [10, 10.5], [100, 100], [0, 0.5]])   # duplicate and far centroids
    C, f, it, empty = native.lloyd(_t(S), _t(C0), 300, 1e-4)
    ref = okm.lloyd(S, C0, 300, 1e-4)
    assert _eq_f32(C.cpu().numpy(), ref["C"]) and f == ref["f"] and it == ref["iters"]
    assert empty.cpu().numpy().tolist() == [False, False, True, True]


# -------------------------------------------------------------- a9 full pass
@pytest.mark.parametrize("m,n,k", [(1, 2, 1), (4097, 2, 5), (100_003, 16, 25), (65_536, 3, 7),
                                   (30_001, 64, 100), (20_000, 33, 40), (5000, 1, 3)])
def test_assign_bit_exact(m, n, k):
    X = gaussian_mixture(m, n, max(1, k // 2), seed=m + k)
    C = X[np.random.default_rng(k).integers(0, m, k)].copy()
    Y, f, rep = native.assign(_t(X), _t(C))
    lab, dist = okm.assign(X, C)
    assert np.array_equal(Y.cpu().numpy(), lab)
    assert f == okm.exact_sum(dist)
    assert rep["inexact_terms"] == 0


def test_assign_ties_lowest_index():
    X = np.float32([[0, 0], [1, 1], [5, 5], [2, 2]] * 300)
    C = np.float32([[1, 0], [0, 1], [1, 0], [5, 5], [2, 2], [2, 2]])
    Y, f, rep = native.assign(_t(X), _t(C))
    lab, dist = okm.assign(X, C)
    assert np.array_equal(Y.cpu().numpy(), lab)
    assert f == okm.exact_sum(dist)
    assert rep["rescored_rows"] >= 300            # equidistant rows are re-scored


# ------------------------------------------------------------- Algorithm 1
def _fit_both(X, k, pol, bud, seed):
    C, Y, rep = native.fit(_t(X), k, native.make_policy(**pol), native.make_budget(**bud), seed=seed)
    ref = obm.bigmeans(X, k, pol, bud, seed=seed)
    return C.cpu().numpy(), Y.cpu().numpy(), rep, ref


def _assert_same(C, Y, rep, ref):
    assert rep["accepts"] == len(ref["L"])
    assert rep["L_sum"] == sum(ref["L"])
    assert rep["s_opt"] == ref["s_opt"]
    assert rep["best_worker"] == ref["best_worker"]
    assert _eq_f32(C, ref["C"])
    assert np.array_equal(Y, ref["labels"])
    assert rep["f_full"] == ref["f_full"]
    assert rep["inexact_terms"] == 0


def test_fit_config1_bit_exact():
    """m=10,000, n=2, 5 Gaussians; k=5, 4 workers, sizes {250,500,1000,2000}, 20 passes."""
    X = workload("gmm_10k_n2_k5")
    pol = dict(set=[250, 500, 1000, 2000], workers=4, passes=10)
    bud = dict(rounds=2, max_lloyd=300, tol=1e-4, kpp_candidates=3)
    C, Y, rep, ref = _fit_both(X, 5, pol, bud, seed=2024)
    _assert_same(C, Y, rep, ref)
    assert rep["lloyd_iters"] == ref["log"]["lloyd_iters"]
    assert rep["passes_done"] == 4 * 20


@pytest.mark.parametrize("m,n,k,pol,rounds,seed", [
    (20_000, 16, 25, dict(s_min=1000, s_max=9000, workers=5, passes=3), 2, 1),
    (9_000, 3, 4, dict(s_min=9000, s_max=9000, workers=2, passes=2), 1, 2),      # s = m
    (12_345, 33, 10, dict(s_min=500, s_max=5000, workers=3, passes=2), 2, 3),
    (3_000, 64, 8, dict(s_min=100, s_max=2999, workers=7, passes=2), 2, 4),
    (5_000, 1, 3, dict(s_min=3, s_max=60, workers=2, passes=4), 3, 5),
])
def test_fit_bit_exact(m, n, k, pol, rounds, seed):
    X = gaussian_mixture(m, n, k, seed=seed, cov="aniso" if n <= 16 else "iso", outliers=0.01)
    bud = dict(rounds=rounds, max_lloyd=300, tol=1e-4, kpp_candidates=3)
    C, Y, rep, ref = _fit_both(X, k, pol, bud, seed)
    _assert_same(C, Y, rep, ref)


def test_fit_duplicate_points_and_more_clusters_than_values():
    X = np.repeat(np.float32([[0, 0], [3, 0], [0, 4]]), 200, axis=0)
    pol = dict(s_min=50, s_max=300, workers=3, passes=3)
    bud = dict(rounds=2, max_lloyd=300, tol=1e-4, kpp_candidates=3)
    C, Y, rep, ref = _fit_both(X, 5, pol, bud, seed=9)
    _assert_same(C, Y, rep, ref)


def test_fit_incumbent_trace_and_session():
    X = gaussian_mixture(30_000, 8, 6, seed=31)
    pol = dict(s_min=500, s_max=4000, workers=4, passes=3)
    bud = dict(rounds=3, max_lloyd=300, tol=1e-4, kpp_candidates=3, eval_full_each_round=True)
    sess = native.FitSession(_t(X), 6, native.make_policy(**pol), native.make_budget(**bud), seed=8)
    sess.rounds(1)
    sess.rounds(2)
    C, Y, rep = sess.finish()
    sess.close()
    ref = obm.bigmeans(X, 6, pol, bud, seed=8)
    _assert_same(C.cpu().numpy(), Y.cpu().numpy(), rep, ref)
    assert rep["f_incumbent"] == min(min(e[3] for e in ref["log"]["incumbent"]), ref["f_full"])


def test_fit_host_buffers_match_device():
    X = gaussian_mixture(8000, 4, 5, seed=3)
    pol = native.make_policy(s_min=300, s_max=3000, workers=3, passes=2)
    bud = native.make_budget(rounds=2)
    C1, Y1, r1 = native.fit(_t(X), 5, pol, bud, seed=11)
    C2, Y2, r2 = native.fit_host(X, 5, pol, bud, seed=11)
    assert _eq_f32(C1.cpu().numpy(), C2) and np.array_equal(Y1.cpu().numpy(), Y2)
    assert r1["f_full"] == r2["f_full"]


def test_errors_are_reported():
    X = _t(gaussian_mixture(100, 2, 2, seed=1))
    with pytest.raises(native.BigmeansError) as e:
        native.fit(X, 5, native.make_policy(s_min=2, s_max=50, workers=2, passes=1),
                   native.make_budget(rounds=1))
    assert e.value.status == native.BM_EINVAL
    Xbad = X.clone()
    Xbad[3, 1] = float("nan")
    with pytest.raises(native.BigmeansError) as e:
        native.fit(Xbad, 2, native.make_policy(s_min=10, s_max=50, workers=2, passes=1),
                   native.make_budget(rounds=1))
    assert e.value.status == native.BM_EINVAL
    with pytest.raises(native.BigmeansError):
        native.sample(1, 3, 0, 0, 0, 10, 11)


# ---------------------------------------------------- full-size configuration
@pytest.mark.slow
def test_config2_full_size_sampled():
    """m=1e6, n=16, k=25, 16 workers, s in [1000, 64000]: one round, then the
    oracle re-derives labels on sampled rows and f(C, X) for the GPU's C."""
    X = workload("gmm_1m_n16_k25")
    pol = native.make_policy(s_min=1000, s_max=64000, workers=16, passes=10)
    bud = native.make_budget(rounds=1, eval_full_each_round=True)
    Xd = _t(X)
    C, Y, rep = native.fit(Xd, 25, pol, bud, seed=7)
    C = C.cpu().numpy()
    Y = Y.cpu().numpy()
    rows = np.random.default_rng(0).integers(0, X.shape[0], 20000)
    lab, _ = okm.assign(X[rows], C)
    assert np.array_equal(Y[rows], lab)
    assert rep["f_full"] == okm.objective(X, C)
    Y2, f2, _ = native.assign(Xd, _t(C))
    assert f2 == rep["f_full"] and np.array_equal(Y2.cpu().numpy(), Y)
    assert rep["inexact_terms"] == 0
    assert rep["passes_done"] == 160


# ------------------------------------------------- size policies (NEXT-4)
@pytest.mark.parametrize("pol,rounds,seed", [
    (dict(s_min=200, s_max=6000, workers=4, passes=2, kind=1), 2, 11),
    (dict(s_min=200, s_max=6000, workers=3, passes=2, exploit=60), 3, 12),
    (dict(s_min=150, s_max=3000, workers=3, passes=2, kind=1, exploit=100), 3, 13),
    (dict(set=[300, 900, 2700], workers=3, passes=2, exploit=50), 3, 14),
])
def test_fit_size_policies_bit_exact(pol, rounds, seed):
    X = gaussian_mixture(8000, 8, 6, seed=seed)
    bud = dict(rounds=rounds, max_lloyd=300, tol=1e-4, kpp_candidates=3)
    C, Y, rep, ref = _fit_both(X, 6, pol, bud, seed=seed)
    _assert_same(C, Y, rep, ref)
    assert rep["lloyd_iters"] == ref["log"]["lloyd_iters"]


# ------------------------------------------- cluster tile (autotuner knob)
def test_results_do_not_depend_on_the_cluster_tile():
    X = gaussian_mixture(60_000, 16, 12, seed=31)
    pol = dict(s_min=3000, s_max=40_000, workers=4, passes=2, kind=1)
    bud = dict(rounds=2, max_lloyd=300, tol=1e-4, kpp_candidates=3)
    outs = []
    try:
        for rows in (512, 0, 8192):
            native.set_rows_per_cta(rows)
            outs.append(native.fit(_t(X), 12, native.make_policy(**pol), native.make_budget(**bud), seed=3))
    finally:
        native.set_rows_per_cta(0)
    (C0, Y0, r0) = outs[0]
    for C, Y, r in outs[1:]:
        assert torch.equal(C.view(torch.int32), C0.view(torch.int32)) and torch.equal(Y, Y0)
        assert r["f_full"] == r0["f_full"] and r["lloyd_iters"] == r0["lloyd_iters"]
    ref = obm.bigmeans(X, 12, pol, bud, seed=3)
    _assert_same(C0.cpu().numpy(), Y0.cpu().numpy(), r0, ref)


def test_autotuner_picks_a_candidate_and_sets_it():
    X = gaussian_mixture(80_000, 32, 10, seed=32)
    pol = native.make_policy(s_min=2000, s_max=50_000, workers=6, passes=2, kind=1)
    try:
        best, ms = native.autotune_rows_per_cta(_t(X), 10, pol, native.make_budget(rounds=2), seed=1,
                                                candidates=(1024, 4096))
        assert best in (1024, 4096) and native.get_rows_per_cta() == best
        assert all(v > 0 for v in ms.values()) and ms[best] == min(ms.values())
    finally:
        native.set_rows_per_cta(0)
    assert native.get_rows_per_cta() == 1024


def test_results_do_not_depend_on_big_cluster_ctas():
    X = gaussian_mixture(200_000, 16, 10, seed=33)
    pol = dict(s_min=20_000, s_max=60_000, workers=3, passes=2)
    bud = dict(rounds=2, max_lloyd=300, tol=1e-4, kpp_candidates=3)
    outs = []
    try:
        for on in (0, 1):
            native.set_big_clusters(on)
            outs.append(native.fit(_t(X), 10, native.make_policy(**pol), native.make_budget(**bud), seed=4))
    finally:
        native.set_big_clusters(0)
    (C0, Y0, r0), (C1, Y1, r1) = outs
    assert torch.equal(C0.view(torch.int32), C1.view(torch.int32)) and torch.equal(Y0, Y1)
    assert r0["f_full"] == r1["f_full"] and r0["lloyd_iters"] == r1["lloyd_iters"]
    ref = obm.bigmeans(X, 10, pol, bud, seed=4)
    _assert_same(C1.cpu().numpy(), Y1.cpu().numpy(), r1, ref)


# --------------------------------------------- worker groups (one launch)
def test_results_do_not_depend_on_worker_groups():
    """Large samples spread over several clusters that add up their exact
    partial sums in global memory (cooperative launch), or one cluster per
    worker: the same bits, equal to the oracle."""
    X = gaussian_mixture(150_000, 16, 12, seed=34, cov="aniso")
    pol = dict(s_min=2000, s_max=70_000, workers=5, passes=3)
    bud = dict(rounds=3, max_lloyd=300, tol=1e-4, kpp_candidates=3, eval_full_each_round=True)
    outs = []
    try:
        for on in (1, 0):
            native.set_worker_groups(on)
            outs.append(native.fit(_t(X), 12, native.make_policy(**pol), native.make_budget(**bud), seed=6))
    finally:
        native.set_worker_groups(1)
    (C0, Y0, r0), (C1, Y1, r1) = outs
    assert torch.equal(C0.view(torch.int32), C1.view(torch.int32)) and torch.equal(Y0, Y1)
    assert r0["f_full"] == r1["f_full"] and r0["lloyd_iters"] == r1["lloyd_iters"]
    assert r0["f_incumbent"] == r1["f_incumbent"]
    ref = obm.bigmeans(X, 12, pol, bud, seed=6)
    _assert_same(C0.cpu().numpy(), Y0.cpu().numpy(), r0, ref)


def test_time_budget_with_worker_groups():
    """A wall-clock budget: the lead CTA of each group decides when to stop
    and every cluster of the group follows; the fit ends with a valid result."""
    X = torch.from_numpy(gaussian_mixture(200_000, 8, 6, seed=35)).cuda()
    pol = native.make_policy(s_min=5000, s_max=80_000, workers=4, passes=10)
    bud = native.make_budget(rounds=0, seconds=0.3)
    C, Y, rep = native.fit(X, 6, pol, bud, seed=2)
    assert rep["rounds_done"] >= 1 and np.isfinite(rep["f_full"]) and rep["f_full"] > 0
    assert int(Y.min()) >= 0 and int(Y.max()) < 6


def test_batched_fits_in_one_launch_equal_the_oracle():
    """Workload-3 shape, reduced: three groups of competing workers with
    k = 10 / 25 / 50 on one data set (4e6 x 32 rows cut to 2e5), octave-uniform
    sample sizes; every round of all three fits runs in one worker launch
    (bm_fit_rounds_batch).  Each group equals its own oracle run."""
    X = workload("gmm_4m_n32_k50o", m=200_000)
    Xd = _t(X)
    groups = ((10, 3), (25, 2), (50, 2))
    bud = dict(rounds=2, max_lloyd=300, tol=1e-4, kpp_candidates=3)
    pols = {k: dict(s_min=2000, s_max=20_000, workers=W, passes=2, kind=1) for k, W in groups}
    sess = [native.FitSession(Xd, k, native.make_policy(**pols[k]), native.make_budget(**bud), seed=300 + k)
            for k, _ in groups]
    native.rounds_batch(sess, 1)
    native.rounds_batch(sess, 1)
    for s_, (k, _) in zip(sess, groups):
        C, Y, rep = s_.finish()
        s_.close()
        ref = obm.bigmeans(X, k, pols[k], bud, seed=300 + k)
        _assert_same(C.cpu().numpy(), Y.cpu().numpy(), rep, ref)
        assert rep["lloyd_iters"] == ref["log"]["lloyd_iters"]


def test_batched_fits_reject_mixed_widths():
    X = _t(gaussian_mixture(20_000, 8, 4, seed=36))
    X2 = _t(gaussian_mixture(20_000, 20, 4, seed=37))
    pol = native.make_policy(s_min=500, s_max=4000, workers=2, passes=1)
    a = native.FitSession(X, 4, pol, native.make_budget(rounds=1), seed=1)
    b = native.FitSession(X2, 4, pol, native.make_budget(rounds=1), seed=1)
    with pytest.raises(native.BigmeansError) as e:
        native.rounds_batch([a, b], 1)
    assert e.value.status == native.BM_EINVAL
    a.close()
    b.close()


# ------------------------------------- a fit sharded over ranks (emulated)
def test_sharded_fit_equals_the_unsharded_fit():
    """Two shards of one fit run one after the other on this GPU (each a rank's
    part: bm_fit_set_workers), combined as the ranks' exchange would (sum of
    L, least f_hat on the common sample, the winner's centroids, full pass):
    the same s_opt, best worker, C, labels and f as the unsharded fit."""
    from paper_2403_18766_gb300 import shard
    X = gaussian_mixture(60_000, 16, 8, seed=38, cov="aniso")
    Xd = _t(X)
    pol = dict(s_min=2000, s_max=30_000, workers=5, passes=3)
    bud = dict(rounds=2, max_lloyd=300, tol=1e-4, kpp_candidates=3)
    C0, Y0, r0 = native.fit(Xd, 8, native.make_policy(**pol), native.make_budget(**bud), seed=9)
    shards = []
    for rank in (0, 1):
        w0, w1 = shard.worker_range(pol["workers"], rank, 2)
        sess = native.FitSession(Xd, 8, native.make_policy(**pol), native.make_budget(**bud), seed=9)
        sess.set_workers(w0, w1)
        sess.rounds(bud["rounds"])
        shards.append((sess, w0, w1, sess.report()))
    L_sum = sum(s[3]["L_sum"] for s in shards)
    L_len = sum(s[3]["accepts"] for s in shards)
    assert L_sum == r0["L_sum"] and L_len == r0["accepts"]
    s_opt = shard.s_opt_from(L_sum, L_len, *shard.size_range(pol, X.shape[0]))
    assert s_opt == r0["s_opt"]
    pairs = []
    for sess, w0, w1, _ in shards:
        pairs += [(v, w0 + i) for i, v in enumerate(sess.recheck(s_opt))]
    f_best, w_best = shard.least(pairs)
    assert w_best == r0["best_worker"]
    owner = next(s for s in shards if s[1] <= w_best < s[2])[0]
    C = owner.worker_centroids(w_best)
    for s in shards:
        s[0].close()
    Y, f, _ = native.assign(Xd, C)
    assert torch.equal(C.view(torch.int32), C0.view(torch.int32))
    assert torch.equal(Y, Y0) and f == r0["f_full"]
    with pytest.raises(native.BigmeansError):           # a shard does not finish on its own
        sess = native.FitSession(Xd, 8, native.make_policy(**pol), native.make_budget(**bud), seed=9)
        sess.set_workers(0, 2)
        sess.rounds(1)
        try:
            sess.finish()
        finally:
            sess.close()
