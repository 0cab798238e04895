"""Thin Python binding of libbigmeans (include/bigmeans.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device buffers are torch tensors (PyTorch provides memory and
streams); they are passed to the C ABI as raw pointers.  If the compiled
library is missing this module raises at import -- there is no CPU path.
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbigmeans.so")

BM_OK, BM_EINVAL, BM_ENOMEM, BM_ECUDA, BM_ETIMEOUT, BM_EINTERNAL, BM_EAGAIN = range(7)
STATUS_NAMES = {0: "BM_OK", 1: "BM_EINVAL", 2: "BM_ENOMEM", 3: "BM_ECUDA", 4: "BM_ETIMEOUT",
                5: "BM_EINTERNAL", 6: "BM_EAGAIN"}
RNG_SIZE, RNG_EVAL, RNG_PASS, RNG_KPP, RNG_FINAL = 1, 2, 3, 4, 5


class SamplePolicy(ctypes.Structure):
    _fields_ = [("s_min", ctypes.c_int64), ("s_max", ctypes.c_int64),
                ("set", ctypes.c_int64 * 16), ("set_len", ctypes.c_int32),
                ("workers", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("kind", ctypes.c_int32), ("exploit", ctypes.c_int32)]


class Budget(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("seconds", ctypes.c_double),
                ("max_lloyd", ctypes.c_int32), ("tol", ctypes.c_double),
                ("kpp_candidates", ctypes.c_int32), ("eval_full_each_round", ctypes.c_int32)]


class Report(ctypes.Structure):
    _fields_ = [("f_full", ctypes.c_double), ("f_incumbent", ctypes.c_double),
                ("s_opt", ctypes.c_int64), ("best_worker", ctypes.c_int32),
                ("rounds_done", ctypes.c_int32), ("passes_done", ctypes.c_int64),
                ("lloyd_iters", ctypes.c_int64), ("assign_rows", ctypes.c_int64),
                ("accepts", ctypes.c_int64), ("L_sum", ctypes.c_int64),
                ("rescored_rows", ctypes.c_int64), ("inexact_terms", ctypes.c_int64),
                ("t_total_s", ctypes.c_double), ("t_worker_s", ctypes.c_double),
                ("t_fullpass_s", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("fullpass_launches", ctypes.c_int64), ("reseeded", ctypes.c_int64),
                ("trace_cycles", ctypes.c_int64 * 16), ("t_sample_s", ctypes.c_double),
                ("t_h2d_s", ctypes.c_double)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["trace_cycles"] = list(d["trace_cycles"])
        return d


class Job(ctypes.Structure):
    _fields_ = [("X_host", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int32),
                ("k", ctypes.c_int32), ("policy", SamplePolicy), ("budget", Budget),
                ("seed", ctypes.c_uint64), ("C_out_host", ctypes.c_void_p),
                ("labels_out_host", ctypes.c_void_p), ("storage", ctypes.c_int32), ("tau", ctypes.c_float)]


class JobResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("state", ctypes.c_int32), ("f_full", ctypes.c_double),
                ("s_opt", ctypes.c_int64), ("t_submit_s", ctypes.c_double), ("t_admit_s", ctypes.c_double),
                ("t_done_s", ctypes.c_double), ("footprint_bytes", ctypes.c_int64), ("report", Report)]


class CtxInfo(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("in_use_bytes", ctypes.c_int64),
                ("peak_in_use_bytes", ctypes.c_int64), ("active", ctypes.c_int32),
                ("peak_active", ctypes.c_int32), ("queued", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("done", ctypes.c_int64), ("now_s", ctypes.c_double)]


class BigmeansError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'`")
lib = ctypes.CDLL(LIB_PATH)

_p = ctypes.c_void_p
_i32, _i64, _u64, _dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
_PP, _BP, _RP = ctypes.POINTER(SamplePolicy), ctypes.POINTER(Budget), ctypes.POINTER(Report)

# Every symbol include/bigmeans.h declares, with its signature.
SIGNATURES = {
    "bigmeans_fit": (_i32, [_p, _i64, _i32, _i32, _PP, _BP, _u64, _p, _p, _p, _RP]),
    "bigmeans_fit_dt": (_i32, [_p, _p, _i32, _i64, _i32, _i32, _PP, _BP, _u64, _i32, _p, _p, _p, _RP]),
    "bm_fit_state_size": (_i32, [_p, ctypes.POINTER(_i64)]),
    "bm_fit_export": (_i32, [_p, _p, _i64]),
    "bm_fit_import": (_i32, [_p, _p, _i64]),
    "bigmeans_fit_host": (_i32, [_p, _i64, _i32, _i32, _PP, _BP, _u64, _p, _p, _p, _RP]),
    "bm_fit_create": (_i32, [_p, _i64, _i32, _i32, _PP, _BP, _u64, _p, ctypes.POINTER(_p)]),
    "bm_fit_rounds": (_i32, [_p, _i32]),
    "bm_fit_rounds_batch": (_i32, [ctypes.POINTER(_p), _i32, _i32]),
    "bm_fit_set_workers": (_i32, [_p, _i32, _i32]),
    "bm_fit_recheck": (_i32, [_p, _i64, ctypes.POINTER(_dbl)]),
    "bm_fit_worker_centroids": (_i32, [_p, _i32, _p]),
    "bm_fit_finish": (_i32, [_p, _p, _p, _RP]),
    "bm_fit_destroy": (None, [_p]),
    "bm_fit_report": (_i32, [_p, _RP]),
    "bm_sample": (_i32, [_u64, _i32, _i32, _i32, _i32, _i64, _i64, _p, _p]),
    "bm_gather": (_i32, [_p, _i64, _i32, _p, _i64, _p, _p]),
    "bm_kmeanspp": (_i32, [_p, _i64, _i32, _p, _i32, _p, _i32, _u64, _i32, _i32, _i32, _p]),
    "bm_lloyd": (_i32, [_p, _i64, _i32, _p, _i32, _i32, _dbl, ctypes.POINTER(_dbl),
                        ctypes.POINTER(_i32), _p, _p]),
    "bm_assign": (_i32, [_p, _i64, _i32, _p, _i32, _p, ctypes.POINTER(_dbl), _RP, _p]),
    "bm_assign_noalloc": (_i32, [_p, _i64, _i32, _p, _i32, _p, ctypes.POINTER(_dbl), _p]),
    "bm_pack_bf16": (_i32, [_p, _i64, _i32, _p, _p, _p]),
    "bm_assign_bf16": (_i32, [_p, _p, _p, _i64, _i32, _p, _i32, ctypes.c_float, _p,
                              ctypes.POINTER(_dbl), _RP, _p]),
    "bm_assign_bf16_certified": (_i32, [_p, _p, _p, _i64, _i32, _p, _i32, ctypes.c_float, _p,
                              ctypes.POINTER(_dbl), _RP, _p]),
    "bm_set_fullpass_impl": (_i32, [_i32]),
    "bm_debug_fail_allocs": (_i32, [_i32]),
    "bm_debug_set_wait_limit": (_i32, [ctypes.c_uint32, ctypes.c_uint32]),
    "bm_last_fullpass_impl": (_i32, []),
    "bm_fit_footprint": (_i32, [_i64, _i32, _i32, _PP, _BP, ctypes.POINTER(_i64)]),
    "bm_set_rows_per_cta": (_i32, [_i32]),
    "bm_trim_memory": (_i32, []),
    "bm_set_big_clusters": (_i32, [_i32]),
    "bm_set_worker_groups": (_i32, [_i32]),
    "bm_get_worker_groups": (_i32, []),
    "bm_get_big_clusters": (_i32, []),
    "bm_set_sampler_impl": (_i32, [_i32]),
    "bm_get_sampler_impl": (_i32, []),
    "bm_get_rows_per_cta": (_i32, []),
    "bm_autotune_rows_per_cta": (_i32, [_p, _i64, _i32, _i32, _PP, _BP, _u64, _p, ctypes.POINTER(_i32), _i32,
                                        ctypes.POINTER(_i32), ctypes.POINTER(_dbl)]),
    "bm_ctx_create": (_i32, [_i64, _i32, ctypes.POINTER(_p)]),
    "bm_job_footprint": (_i32, [ctypes.POINTER(Job), ctypes.POINTER(_i64)]),
    "bm_submit": (_i32, [_p, ctypes.POINTER(Job), ctypes.POINTER(_i64)]),
    "bm_poll": (_i32, [_p, _i64, ctypes.POINTER(JobResult)]),
    "bm_wait": (_i32, [_p, _i64, _dbl, ctypes.POINTER(JobResult)]),
    "bm_job_error": (_i32, [_p, _i64, ctypes.c_char_p, _i64]),
    "bm_ctx_stats": (_i32, [_p, ctypes.POINTER(CtxInfo)]),
    "bm_ctx_destroy": (None, [_p]),
    "bm_last_error": (ctypes.c_char_p, []),
    "bm_version": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in SIGNATURES.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _check(status):
    if status != BM_OK:
        raise BigmeansError(status, lib.bm_last_error().decode())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_f32(t, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32):
        raise TypeError(f"{name} must be a CUDA float32 tensor")
    return t.contiguous()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def make_policy(s_min=None, s_max=None, sizes=None, workers=4, passes=10, set=None, kind=0, exploit=0):
    """bm_sample_policy: a size range [s_min, s_max] or a set of sizes (`sizes` or `set`);
    kind 0 = uniform, 1 = octave-uniform over the range; exploit = percent chance of
    using the rounded mean of L so far."""
    pol = SamplePolicy()
    sizes = sizes if sizes is not None else set
    if sizes:
        sizes = list(sizes)
        assert 1 <= len(sizes) <= 16
        for i, v in enumerate(sizes):
            pol.set[i] = int(v)
        pol.set_len = len(sizes)
        pol.s_min, pol.s_max = min(sizes), max(sizes)
    else:
        pol.s_min, pol.s_max, pol.set_len = int(s_min), int(s_max), 0
    pol.workers, pol.passes = int(workers), int(passes)
    pol.kind, pol.exploit = int(kind), int(exploit)
    return pol


def make_budget(rounds=2, seconds=0.0, max_lloyd=300, tol=1e-4, kpp_candidates=3,
                eval_full_each_round=False):
    b = Budget()
    b.rounds, b.seconds, b.max_lloyd, b.tol = int(rounds), float(seconds), int(max_lloyd), float(tol)
    b.kpp_candidates, b.eval_full_each_round = int(kpp_candidates), int(bool(eval_full_each_round))
    return b


def fit(X, k, policy, budget, seed=0, labels=True, stream=None):
    """bigmeans_fit on a CUDA tensor X (m x n).  Returns (C, labels|None, report)."""
    X = _dev_f32(X, "X")
    m, n = X.shape
    C = torch.empty((k, n), dtype=torch.float32, device=X.device)
    Y = torch.empty(m, dtype=torch.int32, device=X.device) if labels else None
    rep = Report()
    _check(lib.bigmeans_fit(_ptr(X), m, n, k, ctypes.byref(policy), ctypes.byref(budget), seed,
                            _stream(stream), _ptr(C), _ptr(Y), ctypes.byref(rep)))
    return C, Y, rep.as_dict()


BM_F32, BM_BF16 = 0, 1
BM_MODE_EXACT, BM_MODE_FAST = 0, 1


def fit_dt(X, k, policy, budget, seed=0, mode=BM_MODE_EXACT, labels=True, stream=None):
    """bigmeans_fit_dt.  X: a CUDA float32 tensor (BM_F32) or a PackedBF16
    (BM_BF16, its FP32 master as X_master).  mode: BM_MODE_EXACT or
    BM_MODE_FAST.  Returns (C, labels|None, report)."""
    if isinstance(X, PackedBF16):
        Xd, Xm, dt = X.Xb, X.X, BM_BF16
    else:
        Xd = _dev_f32(X, "X")
        Xm, dt = None, BM_F32
    master = Xm if Xm is not None else Xd
    m, n = master.shape
    C = torch.empty((k, n), dtype=torch.float32, device=master.device)
    Y = torch.empty(m, dtype=torch.int32, device=master.device) if labels else None
    rep = Report()
    _check(lib.bigmeans_fit_dt(_ptr(Xd), _ptr(Xm), dt, m, n, k, ctypes.byref(policy), ctypes.byref(budget), seed,
                               int(mode), _stream(stream), _ptr(C), _ptr(Y), ctypes.byref(rep)))
    return C, Y, rep.as_dict()


def fit_host(X, k, policy, budget, seed=0, labels=True, stream=None):
    """bigmeans_fit_host on host memory (numpy or CPU tensor); copies happen inside."""
    Xn = np.ascontiguousarray(X.numpy() if isinstance(X, torch.Tensor) else X, dtype=np.float32)
    m, n = Xn.shape
    C = np.empty((k, n), dtype=np.float32)
    Y = np.empty(m, dtype=np.int32) if labels else None
    rep = Report()
    _check(lib.bigmeans_fit_host(Xn.ctypes.data_as(_p), m, n, k, ctypes.byref(policy),
                                 ctypes.byref(budget), seed, _stream(stream),
                                 C.ctypes.data_as(_p),
                                 Y.ctypes.data_as(_p) if Y is not None else _p(0),
                                 ctypes.byref(rep)))
    return C, Y, rep.as_dict()


class FitSession:
    """Staged fit (bm_fit_create / bm_fit_rounds / bm_fit_finish)."""

    def __init__(self, X, k, policy, budget, seed=0, stream=None):
        self.X = _dev_f32(X, "X")
        self.k = k
        self.stream = stream
        self.ctx = ctypes.c_void_p(0)
        m, n = self.X.shape
        _check(lib.bm_fit_create(_ptr(self.X), m, n, k, ctypes.byref(policy), ctypes.byref(budget),
                                 seed, _stream(stream), ctypes.byref(self.ctx)))

    def rounds(self, r):
        _check(lib.bm_fit_rounds(self.ctx, int(r)))

    def finish(self, labels=True):
        m, n = self.X.shape
        C = torch.empty((self.k, n), dtype=torch.float32, device=self.X.device)
        Y = torch.empty(m, dtype=torch.int32, device=self.X.device) if labels else None
        rep = Report()
        _check(lib.bm_fit_finish(self.ctx, _ptr(C), _ptr(Y), ctypes.byref(rep)))
        return C, Y, rep.as_dict()

    def report(self):
        rep = Report()
        _check(lib.bm_fit_report(self.ctx, ctypes.byref(rep)))
        return rep.as_dict()

    def export_state(self):
        """bm_fit_export: the fit's state between rounds, as bytes."""
        n = _i64(0)
        _check(lib.bm_fit_state_size(self.ctx, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(int(n.value))
        _check(lib.bm_fit_export(self.ctx, buf, n.value))
        return buf.raw

    def import_state(self, state):
        """bm_fit_import: continue from a state exported by another session of the same fit."""
        buf = ctypes.create_string_buffer(bytes(state), len(state))
        _check(lib.bm_fit_import(self.ctx, buf, len(state)))

    def set_workers(self, w_begin, w_end):
        """bm_fit_set_workers: run only workers [w_begin, w_end) (a shard of the fit)."""
        _check(lib.bm_fit_set_workers(self.ctx, int(w_begin), int(w_end)))
        self.w_range = (int(w_begin), int(w_end))

    def recheck(self, s_opt):
        """bm_fit_recheck: f_hat of the shard's workers on the common sample of size s_opt."""
        w0, w1 = getattr(self, "w_range", (0, None))
        if w1 is None:
            raise ValueError("set_workers first")
        f = (ctypes.c_double * (w1 - w0))()
        _check(lib.bm_fit_recheck(self.ctx, int(s_opt), f))
        return list(f)

    def worker_centroids(self, w):
        """bm_fit_worker_centroids: worker w's centroids (k x n, device)."""
        m, n = self.X.shape
        C = torch.empty((self.k, n), dtype=torch.float32, device=self.X.device)
        _check(lib.bm_fit_worker_centroids(self.ctx, int(w), _ptr(C)))
        return C

    def close(self):
        if self.ctx:
            lib.bm_fit_destroy(self.ctx)
            self.ctx = ctypes.c_void_p(0)

    def __del__(self):
        self.close()


def rounds_batch(sessions, r):
    """bm_fit_rounds_batch: the next r rounds of several FitSessions, every
    round of all of them in one worker launch (on the first session's stream)."""
    arr = (ctypes.c_void_p * len(sessions))(*[sess.ctx.value for sess in sessions])
    _check(lib.bm_fit_rounds_batch(arr, len(sessions), int(r)))


def sample(seed, purpose, worker, rnd, pss, m, s, device="cuda", stream=None):
    out = torch.empty(max(int(s), 1), dtype=torch.int64, device=device)
    _check(lib.bm_sample(seed, purpose, worker, rnd, pss, m, s, _ptr(out), _stream(stream)))
    return out[: int(s)]


def gather(X, idx, stream=None):
    X = _dev_f32(X, "X")
    idx = idx.to(torch.int64).contiguous()
    S = torch.empty((idx.numel(), X.shape[1]), dtype=torch.float32, device=X.device)
    _check(lib.bm_gather(_ptr(X), X.shape[0], X.shape[1], _ptr(idx), idx.numel(), _ptr(S),
                         _stream(stream)))
    return S


def kmeanspp(S, C, degenerate, trials, seed, worker, rnd, pss, stream=None):
    S = _dev_f32(S, "S")
    C = _dev_f32(C, "C").clone()
    deg = torch.as_tensor(degenerate, dtype=torch.uint8, device=S.device).contiguous()
    _check(lib.bm_kmeanspp(_ptr(S), S.shape[0], S.shape[1], _ptr(C), C.shape[0], _ptr(deg), trials,
                           seed, worker, rnd, pss, _stream(stream)))
    return C


def lloyd(S, C, max_iter=300, tol=1e-4, stream=None):
    S = _dev_f32(S, "S")
    C = _dev_f32(C, "C").clone()
    empty = torch.empty(C.shape[0], dtype=torch.uint8, device=S.device)
    f = ctypes.c_double(0)
    it = ctypes.c_int32(0)
    _check(lib.bm_lloyd(_ptr(S), S.shape[0], S.shape[1], _ptr(C), C.shape[0], max_iter, tol,
                        ctypes.byref(f), ctypes.byref(it), _ptr(empty), _stream(stream)))
    return C, f.value, it.value, empty.bool()


def assign(X, C, labels=True, stream=None):
    X = _dev_f32(X, "X")
    C = _dev_f32(C, "C")
    Y = torch.empty(X.shape[0], dtype=torch.int32, device=X.device) if labels else None
    f = ctypes.c_double(0)
    rep = Report()
    _check(lib.bm_assign(_ptr(X), X.shape[0], X.shape[1], _ptr(C), C.shape[0], _ptr(Y),
                         ctypes.byref(f), ctypes.byref(rep), _stream(stream)))
    return Y, f.value, rep.as_dict()


def set_fullpass_impl(impl):
    """bm_set_fullpass_impl: 0 = by shape, 1 = FP32-ALU pass, 2 = tensor-core pass where it applies."""
    _check(lib.bm_set_fullpass_impl(int(impl)))


def last_fullpass_impl():
    """bm_last_fullpass_impl: 2 = tensor cores, 1 = FP32 ALU, 0 = none yet (this thread)."""
    return int(lib.bm_last_fullpass_impl())


def assign_noalloc(X, C, labels=True, stream=None):
    """bm_assign_noalloc: the full-data pass using the library's fixed scratch
    (no device allocation inside the call); calls must not overlap on the GPU."""
    X = _dev_f32(X, "X")
    C = _dev_f32(C, "C")
    Y = torch.empty(X.shape[0], dtype=torch.int32, device=X.device) if labels else None
    f = ctypes.c_double(0)
    _check(lib.bm_assign_noalloc(_ptr(X), X.shape[0], X.shape[1], _ptr(C), C.shape[0], _ptr(Y),
                                 ctypes.byref(f), _stream(stream)))
    return Y, f.value


class PackedBF16:
    """X packed for the tensor-core full pass (bm_pack_bf16); keeps the FP32 master."""

    def __init__(self, X, stream=None):
        self.X = _dev_f32(X, "X")
        m, n = self.X.shape
        m_pad = (m + 127) // 128 * 128
        # 1024-byte aligned buffer carved from a larger allocation
        self._raw = torch.empty(m_pad * 128 + 1024, dtype=torch.uint8, device=self.X.device)
        off = (-self._raw.data_ptr()) % 1024
        self.Xb = self._raw[off:off + m_pad * 128]
        self.norms = torch.empty(m_pad + 1, dtype=torch.float32, device=self.X.device)
        _check(lib.bm_pack_bf16(_ptr(self.X), m, n, _ptr(self.Xb), _ptr(self.norms), _stream(stream)))


def assign_bf16(packed, C, tau=1e-3, labels=True, stream=None, certified=False):
    """bm_assign_bf16 (or bm_assign_bf16_certified): precision-form full pass on tensor cores."""
    C = _dev_f32(C, "C")
    X = packed.X
    Y = torch.empty(X.shape[0], dtype=torch.int32, device=X.device) if labels else None
    f = ctypes.c_double(0)
    rep = Report()
    fn = lib.bm_assign_bf16_certified if certified else lib.bm_assign_bf16
    _check(fn(_ptr(packed.Xb), _ptr(packed.norms), _ptr(X), X.shape[0], X.shape[1],
              _ptr(C), C.shape[0], float(tau), _ptr(Y), ctypes.byref(f),
              ctypes.byref(rep), _stream(stream)))
    return Y, f.value, rep.as_dict()


def version():
    return lib.bm_version().decode()


def fit_footprint(m, n, k, policy, budget):
    """bm_fit_footprint: device bytes of a fit's workspace."""
    b = ctypes.c_int64(0)
    _check(lib.bm_fit_footprint(int(m), int(n), int(k), ctypes.byref(policy), ctypes.byref(budget), ctypes.byref(b)))
    return b.value


class ServeContext:
    """Serving context (bm_ctx_*): jobs admitted by device-memory footprint and
    run concurrently.  Host buffers of a job are kept referenced until it is done."""

    def __init__(self, hbm_budget_bytes, max_active=4):
        self.ctx = ctypes.c_void_p(0)
        _check(lib.bm_ctx_create(int(hbm_budget_bytes), int(max_active), ctypes.byref(self.ctx)))
        self._keep = {}

    def submit(self, X, k, policy, budget, seed=0, labels=True, bf16=False, tau=1e-3):
        """X: host float32 array (numpy or CPU tensor, pinned preferred). bf16: also hold X packed
        in BF16 and take labels and f from the precision pass (tau). Returns the job id."""
        if isinstance(X, torch.Tensor):
            Xt = X.contiguous()
            assert Xt.device.type == "cpu" and Xt.dtype == torch.float32
            m, n = Xt.shape
            xptr = Xt.data_ptr()
        else:
            Xt = np.ascontiguousarray(X, dtype=np.float32)
            m, n = Xt.shape
            xptr = Xt.ctypes.data
        pin = torch.cuda.is_available()
        C = torch.empty((k, n), dtype=torch.float32, pin_memory=pin)
        Y = torch.empty(m, dtype=torch.int32, pin_memory=pin) if labels else None
        job = Job(X_host=xptr, m=m, n=n, k=k, policy=policy, budget=budget, seed=seed,
                  C_out_host=C.data_ptr(), labels_out_host=(Y.data_ptr() if Y is not None else 0),
                  storage=1 if bf16 else 0, tau=float(tau))
        jid = ctypes.c_int64(0)
        _check(lib.bm_submit(self.ctx, ctypes.byref(job), ctypes.byref(jid)))
        self._keep[jid.value] = (Xt, C, Y, job)
        return jid.value

    def _result(self, jid, res):
        d = {name: getattr(res, name) for name, _ in res._fields_ if name != "report"}
        d["report"] = res.report.as_dict()
        if res.state == 2:
            Xt, C, Y, _ = self._keep[jid]
            d["C"], d["labels"] = C, Y
            if res.status != BM_OK:
                buf = ctypes.create_string_buffer(512)
                lib.bm_job_error(self.ctx, jid, buf, 512)
                d["error"] = buf.value.decode()
        return d

    def poll(self, jid):
        res = JobResult()
        st = lib.bm_poll(self.ctx, int(jid), ctypes.byref(res))
        if st not in (BM_OK, BM_EAGAIN):
            _check(st)
        return self._result(jid, res)

    def wait(self, jid, timeout=None):
        res = JobResult()
        st = lib.bm_wait(self.ctx, int(jid), -1.0 if timeout is None else float(timeout), ctypes.byref(res))
        if st not in (BM_OK, BM_EAGAIN):
            _check(st)
        return self._result(jid, res)

    def stats(self):
        info = CtxInfo()
        _check(lib.bm_ctx_stats(self.ctx, ctypes.byref(info)))
        return {name: getattr(info, name) for name, _ in info._fields_ if name != "pad_"}

    def close(self):
        if self.ctx:
            lib.bm_ctx_destroy(self.ctx)
            self.ctx = ctypes.c_void_p(0)


def set_rows_per_cta(rows):
    """bm_set_rows_per_cta (0 = default)."""
    _check(lib.bm_set_rows_per_cta(int(rows)))


def get_rows_per_cta():
    return int(lib.bm_get_rows_per_cta())


def autotune_rows_per_cta(X, k, policy, budget, seed=0, candidates=(1024, 2048, 4096, 8192), stream=None):
    """bm_autotune_rows_per_cta: times one round per candidate, keeps the fastest.
    Returns (best, {candidate: ms})."""
    X = _dev_f32(X, "X")
    cand = (ctypes.c_int32 * len(candidates))(*[int(c) for c in candidates])
    ms = (ctypes.c_double * len(candidates))()
    best = ctypes.c_int32(0)
    _check(lib.bm_autotune_rows_per_cta(_ptr(X), X.shape[0], X.shape[1], int(k), ctypes.byref(policy),
                                        ctypes.byref(budget), int(seed), _stream(stream), cand, len(candidates),
                                        ctypes.byref(best), ms))
    return best.value, {int(c): float(t) for c, t in zip(candidates, ms)}


def set_big_clusters(on):
    """bm_set_big_clusters: 512-thread CTAs for the workers whose cluster is at the cap."""
    _check(lib.bm_set_big_clusters(int(bool(on))))


def set_worker_groups(on):
    """bm_set_worker_groups: 1 = large samples may span several clusters (cooperative launch), 0 = never."""
    _check(lib.bm_set_worker_groups(int(bool(on))))


def get_worker_groups():
    return int(lib.bm_get_worker_groups())


def get_big_clusters():
    return int(lib.bm_get_big_clusters())


def set_sampler_impl(impl):
    """bm_set_sampler_impl: 0 = shared-memory bitmap where it fits, 1 = device tables."""
    _check(lib.bm_set_sampler_impl(int(impl)))


def get_sampler_impl():
    return int(lib.bm_get_sampler_impl())


def debug_fail_allocs(count):
    """bm_debug_fail_allocs: the next `count` device allocations of the library fail (test hook)."""
    _check(lib.bm_debug_fail_allocs(int(count)))


def debug_set_wait_limit(polls, sleep_ns=0):
    """bm_debug_set_wait_limit: bounded-wait limit of the tensor-core exact pass (0 = default; test hook)."""
    _check(lib.bm_debug_set_wait_limit(int(polls), int(sleep_ns)))


def trim_memory():
    """bm_trim_memory: return the library pool's unused device memory."""
    _check(lib.bm_trim_memory())
