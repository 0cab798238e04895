"""GPU tests of checkpoint/resume of a staged fit (bm_fit_export / bm_fit_import).

A fit that runs r rounds, exports its state, and is continued in a new
context created with the same arguments must end exactly where the
uninterrupted fit ends: the same C_best, labels, f(C, X), s_opt, best worker
and counters (samples, seeds and sizes are functions of (seed, worker, round,
pass)).  Covered for the paper's uniform sizes and for the exploit policy
(sizes drawn from the mean of L, so L itself must be restored), and against
the oracle's Algorithm 1 on the small workload.  A state is refused by a
context of another fit, after a round has run, or when truncated.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import bigmeans as obm  # noqa: E402
from paper_2403_18766_gb300 import native  # noqa: E402
from paper_2403_18766_gb300.synthetic import gaussian_mixture, workload  # noqa: E402


def _keys(rep):
    names = ("f_full", "f_incumbent", "s_opt", "best_worker", "rounds_done", "passes_done", "lloyd_iters",
             "assign_rows", "accepts", "L_sum", "reseeded")
    assert all(k in rep for k in names)
    return {k: rep[k] for k in names}


def _run(X, k, pol, bud, seed, split):
    """(C, Y, report) of a fit of bud rounds, interrupted after `split` rounds
    (None: not interrupted)."""
    T = bud.rounds
    if split is None:
        s = native.FitSession(X, k, pol, bud, seed=seed)
        s.rounds(T)
        out = s.finish()
        s.close()
        return out
    a = native.FitSession(X, k, pol, bud, seed=seed)
    a.rounds(split)
    state = a.export_state()
    a.close()
    b = native.FitSession(X, k, pol, bud, seed=seed)
    b.import_state(state)
    b.rounds(T - split)
    out = b.finish()
    b.close()
    return out


@pytest.mark.parametrize("exploit", [0, 60])
def test_resumed_fit_equals_uninterrupted(exploit):
    X = gaussian_mixture(30_000, 8, 6, seed=51)
    Xd = torch.from_numpy(X).cuda()
    pol = native.make_policy(s_min=600, s_max=5000, workers=4, passes=3, exploit=exploit)
    bud = native.make_budget(rounds=4)
    C0, Y0, r0 = _run(Xd, 6, pol, bud, 7, None)
    for split in (1, 3):
        C1, Y1, r1 = _run(Xd, 6, pol, bud, 7, split)
        assert torch.equal(C0, C1) and torch.equal(Y0, Y1)
        assert _keys(r0) == _keys(r1)


def test_resumed_fit_equals_the_oracle():
    """Workload 1 (10^4 x 2, k = 5): rounds 1 + 1 across an export equal the
    oracle's two-round Algorithm 1."""
    X = workload("gmm_10k_n2_k5")
    policy = dict(set=[250, 500, 1000, 2000], workers=4, passes=10)
    budget = dict(rounds=2, max_lloyd=300, tol=1e-4, kpp_candidates=3)
    ref = obm.bigmeans(X, 5, policy, budget, 2024)
    C, Y, rep = _run(torch.from_numpy(X).cuda(), 5, native.make_policy(**policy), native.make_budget(**budget),
                     2024, 1)
    assert np.array_equal(C.cpu().numpy(), np.asarray(ref["C"], np.float32))
    assert np.array_equal(Y.cpu().numpy(), ref["labels"])
    assert rep["s_opt"] == ref["s_opt"] and rep["best_worker"] == ref["best_worker"]


def test_state_is_refused_by_another_fit():
    X = gaussian_mixture(20_000, 8, 6, seed=53)
    Xd = torch.from_numpy(X).cuda()
    pol = native.make_policy(s_min=600, s_max=4000, workers=4, passes=3)
    bud = native.make_budget(rounds=3)
    a = native.FitSession(Xd, 6, pol, bud, seed=3)
    a.rounds(1)
    state = a.export_state()
    with pytest.raises(native.BigmeansError):          # a round has run in this context
        a.import_state(state)
    a.close()
    others = [native.FitSession(Xd, 6, pol, bud, seed=4),                                    # seed
              native.FitSession(Xd, 7, pol, bud, seed=3),                                    # k
              native.FitSession(Xd, 6, native.make_policy(s_min=600, s_max=4000, workers=4, passes=4), bud,
                                seed=3),                                                     # passes
              native.FitSession(Xd, 6, native.make_policy(s_min=700, s_max=4000, workers=4, passes=3), bud,
                                seed=3),                                                     # size policy
              native.FitSession(Xd * 2, 6, pol, bud, seed=3)]                                # another X
    for o in others:
        with pytest.raises(native.BigmeansError):
            o.import_state(state)
        o.close()
    b = native.FitSession(Xd, 6, pol, bud, seed=3)
    with pytest.raises(native.BigmeansError):          # truncated
        b.import_state(state[:-9])
    with pytest.raises(native.BigmeansError):          # not a state
        b.import_state(b"\0" * len(state))
    b.import_state(state)                               # the right one still loads
    b.rounds(2)
    b.close()
