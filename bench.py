"""Benchmark: competitive-sample-size Big-means on one GB300 (or N, one per rank).

Workload (the configuration the headline metric is quoted on):
  m = 1,000,000 rows, n = 16, mixture of 25 anisotropic Gaussians
  (eigenvalues in [0.1, 4], Dirichlet(1) weights), k = 25, 16 competing
  workers, sample sizes uniform in [1,000, 64,000], p = 10 passes per round,
  Lloyd <= 300 iterations / tol 1e-4, K-means++ with 3 candidates, and the
  full-data f(C, X) of the incumbent after every round.

One step = one round of Algorithm 1 for all workers (f_hat recompute, 10
passes of sample + gather + re-seed + Lloyd + incumbent rule) plus the
full-data pass that evaluates the incumbent.  Metric: Lloyd pts*k/s = (rows
assigned inside Lloyd runs) * k / device time.  L2 is flushed (256 MB write)
between timed steps, outside the timed region.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "gmm_1m_n16_k25"
K_CLUSTERS = 25
POLICY = dict(s_min=1000, s_max=64000, workers=16, passes=10)
BUDGET = dict(max_lloyd=300, tol=1e-4, kpp_candidates=3, eval_full_each_round=True)
METRIC = "Lloyd pts·k/s"
UNIT = "pts·k/s"
FP32_LANES_PER_SM = 128                  # FP32 FMA lanes per SM (4 SMSPs x 32)
NOMINAL_SMS, NOMINAL_MAX_MHZ = 152, 2070.0


def config_dict(m, n):
    return {"workload": f"{WORKLOAD}: m={m}, n={n}, 25 anisotropic Gaussians, k={K_CLUSTERS}, "
                        f"W={POLICY['workers']} workers, s in [{POLICY['s_min']}, {POLICY['s_max']}], "
                        f"p={POLICY['passes']}",
            "m": m, "n": n, "k": K_CLUSTERS, "workers": POLICY["workers"],
            "s_range": [POLICY["s_min"], POLICY["s_max"]], "passes": POLICY["passes"],
            "step": "one Algorithm-1 round (all workers) + full-data pass of the incumbent",
            "l2": "flushed between timed steps (256 MB write), outside the timed region"}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def rank_seed(rank):
    """Seed of the fit: on N ranks one fit of N x 16 workers (each rank runs
    its 16 workers), so every rank uses the same seed."""
    return 1000


def finish_sharded(sess, Xd, k, policy, rank, world):
    """The end of a fit sharded over the ranks (paper_2403_18766_gb300.shard):
    the global mean of L, the common recheck of each rank's workers, the
    least f_hat over all ranks, the winner's centroids broadcast, and the
    full-data pass.  Returns (C, labels, report-like dict)."""
    from paper_2403_18766_gb300 import native, shard
    rep = sess.report()
    m = Xd.shape[0]
    w0, w1 = shard.worker_range(policy["workers"], rank, world)
    L_sum, L_len = shard.global_L(rep["L_sum"], rep["accepts"], None, Xd.device)
    s_opt = shard.s_opt_from(L_sum, L_len, *shard.size_range(policy, m))
    f_best, w_best = shard.pick_best(sess.recheck(s_opt), w0, None, Xd.device)
    owner = next(r for r in range(world)
                 if shard.worker_range(policy["workers"], r, world)[0] <= w_best
                 < shard.worker_range(policy["workers"], r, world)[1])
    C = sess.worker_centroids(w_best) if owner == rank else None
    C = shard.broadcast_centroids(C, owner, (k, Xd.shape[1]), None, Xd.device)
    Y, f, _ = native.assign(Xd, C)
    return C, Y, dict(rep, f_full=f, s_opt=s_opt, best_worker=w_best)


def aggregate(t_local, work_local, device="cpu"):
    """Whole-job numbers over the ranks of the default process group: the
    slowest rank's time and the total work (units all ranks processed).
    Works with any backend (NCCL on GPUs, gloo on CPU)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([float(work_local)], dtype=torch.float64, device=device)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": NOMINAL_MAX_MHZ}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling around the timed region.

    nvidia-smi samples every `interval_ms` (line-buffered through stdbuf where
    available) and stamps each sample itself; a reader thread collects the
    lines.  The constructor waits (up to 3 s) for the first sample, so that
    sampling is running before the timed region starts; begin() and end()
    mark the region on the host clock, and stop() summarises the samples
    stamped inside it (all samples of the run when the region was too short
    to hold one, said by `in_region`)."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device_index, interval_ms=20):
        import shutil
        import threading
        self.proc, self.lines, self.t0, self.t1 = None, [], None, None
        self._first = threading.Event()
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", str(interval_ms), "-i", str(device_index)]
        if shutil.which("stdbuf"):
            cmd = ["stdbuf", "-oL"] + cmd
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self._reader = threading.Thread(target=self._read, daemon=True)
        self._reader.start()
        self._first.wait(timeout=3.0)

    def _read(self):
        for line in self.proc.stdout:
            if line.count(",") >= 9:
                self.lines.append(line.strip())
                self._first.set()

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    @staticmethod
    def _stamp(text):
        from datetime import datetime
        try:
            return datetime.strptime(text.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        self._reader.join(timeout=5)
        rows = [r.split(", ") for r in self.lines]
        rows = [r for r in rows if len(r) >= 10]
        if not rows:
            return None
        inside = []
        if self.t0 is not None and self.t1 is not None:
            inside = [r for r in rows if (self._stamp(r[0]) or -1.0) >= self.t0 - 0.005
                      and (self._stamp(r[0]) or -1.0) <= self.t1 + 0.005]
        use = inside or rows
        sm = [float(r[2]) for r in use if r[2].strip().replace(".", "").isdigit()]
        mx = [float(r[3]) for r in use if r[3].strip().replace(".", "").isdigit()]
        reasons = set()
        for r in use:
            for nm, v in zip(self.REASONS, r[6:10]):
                if v.strip() == "Active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(use), "in_region": bool(inside),
                "region_ms": (self.t1 - self.t0) * 1e3 if self.t0 is not None and self.t1 is not None else None}


def _traffic_for(kernel_sources, workload=None):
    """DRAM bytes per launch from a committed ncu summary, if it matches the
    source (entries keyed by the digest of the sources, and by the workload
    where one kernel has captures of several)."""
    h = hashlib.sha256()
    for p in kernel_sources:
        with open(p, "rb") as fh:
            h.update(fh.read())
    digest = h.hexdigest()[:16]
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            tr = json.load(fh)
    except OSError:
        return None, digest
    ent = tr.get(f"{digest}/{workload}" if workload else digest)
    return (ent if ent else None), digest


def _oracle_worker_run(args):
    """One 1-worker oracle fit of the headline workload (spawned process)."""
    rounds, seed = args
    import time as _t
    from oracle import bigmeans as obm
    from paper_2403_18766_gb300.synthetic import workload
    X = workload(WORKLOAD)
    t0 = _t.perf_counter()
    res = obm.bigmeans(X, K_CLUSTERS, dict(POLICY, workers=1),
                       dict(BUDGET, rounds=rounds, eval_full_each_round=False), seed=seed)
    return res["log"]["pts_k"], _t.perf_counter() - t0


def cpu_baseline(X, seconds_target=20.0, multi=True, checks=None):
    """The oracle as it stands, on a bounded sample of the same workload: one
    worker, p passes per round, rounds doubled until about seconds_target/2,
    on one core; then (multi) one spawned process per worker, up to the
    host's cores, each a 1-worker fit of that many rounds, timed together.
    `checks` (optional) are GPU results to compare with the oracle's all-FP64
    mode (pure64): the headline fit's final C, labels and f(C, X), and the
    precision form on a slice of the 10^7 x 64 workload."""
    from oracle import bigmeans as obm
    from oracle import kmeans as okm
    rounds, res, dt = 1, None, 0.0
    while True:
        pol = dict(POLICY, workers=1)
        t0 = time.perf_counter()
        res = obm.bigmeans(X, K_CLUSTERS, pol, dict(BUDGET, rounds=rounds, eval_full_each_round=False),
                           seed=1)
        dt = time.perf_counter() - t0
        if dt >= seconds_target / 2 or rounds >= 64:
            break
        rounds *= 2
    ptsk = res["log"]["pts_k"]
    out = {"value": ptsk / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"1 worker x {rounds} rounds x {POLICY['passes']} passes of the same workload "
                     f"({res['log']['lloyd_iters']} Lloyd updates, {ptsk:.3g} pts*k; time includes "
                     f"sampling, K-means++, the recheck and the final full pass) in {dt:.1f} s"}
    if multi:
        import multiprocessing as mp
        procs = max(1, min(POLICY["workers"], os.cpu_count() or 1))
        r_each = max(1, rounds // 2)
        ctx = mp.get_context("spawn")
        t0 = time.perf_counter()
        with ctx.Pool(procs) as pool:
            parts = pool.map(_oracle_worker_run, [(r_each, 1 + i) for i in range(procs)])
        wall = time.perf_counter() - t0
        tot = sum(p[0] for p in parts)
        out["multi"] = {"value": tot / wall, "unit": UNIT, "cores": procs, "kind": "oracle",
                        "sample": f"{procs} spawned processes (one per worker, up to the host's cores), each a "
                                  f"1-worker fit of {r_each} rounds x {POLICY['passes']} passes; wall time "
                                  f"{wall:.1f} s including process start and data generation"}
    if checks:
        err = {}
        h = checks.get("headline")
        if h:
            lab64, d64 = okm.assign(X, h["C"], mode="pure64")
            f64 = okm.exact_sum(d64)
            err["headline"] = {"f_rel": abs(h["f"] - f64) / f64,
                               "label_mismatch": int((h["labels"] != lab64).sum()), "rows": int(X.shape[0]),
                               "what": "final C of the timed fit: GPU f(C, X) and labels (exact mode) against "
                                       "the FP64 oracle on the same C, all rows"}
        pr = checks.get("precision")
        if pr:
            _, d64 = okm.assign(pr["X"], pr["C"], mode="pure64")
            f64 = okm.exact_sum(d64)
            err["precision"] = {k2: abs(v - f64) / f64 for k2, v in pr["f"].items()}
            err["precision"]["rows"] = int(pr["X"].shape[0])
            err["precision"]["what"] = ("f(C, X) on the first rows of the 10^7 x 64 workload (C of a short fit "
                                        "on all rows) from each GPU form, against the FP64 oracle")
        out["err_vs_pure64"] = err
    return out


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    from paper_2403_18766_gb300.synthetic import workload
    X = workload(WORKLOAD)
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(X, seconds_target=3.0)
    for _ in range(args.steps):
        vals.append(cpu_baseline(X, seconds_target=6.0))
    v = statistics.median([c["value"] for c in vals])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64/f32 (oracle)", "data": "synthetic",
            "config": config_dict(*X.shape),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    from paper_2403_18766_gb300 import native
    from paper_2403_18766_gb300.synthetic import workload

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    X = workload(WORKLOAD)
    m, n = X.shape
    Xd = torch.from_numpy(X).to(dev)
    stream = torch.cuda.current_stream(dev)
    # on N ranks: one fit of N x W workers, rank r running workers [W r, W (r + 1))
    fit_policy = dict(POLICY, workers=POLICY["workers"] * ws)
    pol = native.make_policy(**fit_policy)
    total_rounds = args.warmup + args.steps
    bud = native.make_budget(rounds=total_rounds, **BUDGET)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    sess = native.FitSession(Xd, K_CLUSTERS, pol, bud, seed=rank_seed(rank))
    if ws > 1:
        sess.set_workers(POLICY["workers"] * rank, POLICY["workers"] * (rank + 1))
    clocks = ClockSampler(local)
    trace = []                                  # (cumulative device s, f_incumbent) after each round
    t_cum = 0.0
    for _ in range(args.warmup):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sess.rounds(1)
        b.record(stream)
        torch.cuda.synchronize(dev)
        t_cum += a.elapsed_time(b) / 1e3
        trace.append((t_cum, sess.report()["f_incumbent"]))
    rep0 = sess.report()
    step_ms = []
    clocks.begin()
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sess.rounds(1)
        b.record(stream)
        torch.cuda.synchronize(dev)
        step_ms.append(a.elapsed_time(b))
        t_cum += step_ms[-1] / 1e3
        trace.append((t_cum, sess.report()["f_incumbent"]))
    clocks.end()
    rep1 = sess.report()
    f_end = trace[-1][1]
    tto = next(((t, i + 1) for i, (t, f) in enumerate(trace) if f <= f_end * (1 + 1e-4)), (None, None))
    clk = clocks.stop()
    if ws > 1:
        C, Y_fin, rep_fin = finish_sharded(sess, Xd, K_CLUSTERS, fit_policy, rank, ws)
    else:
        C, Y_fin, rep_fin = sess.finish(labels=True)
    sess.close()

    t_local = sum(step_ms) / 1e3
    rows = rep1["assign_rows"] - rep0["assign_rows"]
    ptsk_local = rows * K_CLUSTERS
    launches = rep1["kernel_launches"] - rep0["kernel_launches"]
    t_worker = rep1["t_worker_s"] - rep0["t_worker_s"]
    n_worker = args.steps                       # one worker launch (all W workers) per step
    t_full = rep1["t_fullpass_s"] - rep0["t_fullpass_s"]
    n_full = rep1["fullpass_launches"] - rep0["fullpass_launches"]
    if ws > 1:
        t_job, ptsk = aggregate(t_local, ptsk_local, dev)
    else:
        t_job, ptsk = t_local, float(ptsk_local)

    peaks, peak_src = _peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", NOMINAL_MAX_MHZ))
    alu_peak = sm_count * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12        # TFLOP/s
    flops = 2.0 * n * K_CLUSTERS * rows
    achieved = flops / t_worker / 1e12 if t_worker > 0 else 0.0
    srcs = [os.path.join(ROOT, "paper_2403_18766_gb300", "csrc", f)
            for f in ("bm_worker_impl.cuh", "bm_worker.cuh", "bm_device.cuh")]
    traffic, digest = _traffic_for(srcs)
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak if alu_peak else None,
                "traffic": traffic.get("dram_bytes_per_launch") if traffic else None,
                "kernel": "worker_kernel<16>: one launch per round for all W workers (K-means++, Lloyd, "
                          "incumbent rule; large samples as groups of clusters), CUDA events around the "
                          "launch on its stream; the next round's sample_kernel<16> runs beside it on a "
                          "second stream",
                "algorithmic": "2*n*k flops per row assigned inside Lloyd; "
                               f"{flops / max(n_worker, 1):.4g} flops per launch",
                "peak_source": f"{sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {max_mhz:.0f} MHz",
                "source_digest": digest}
    bytes_full = m * n * 4.0
    full_gbs = bytes_full * n_full / t_full / 1e9 if t_full > 0 else 0.0
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    tensor_full = native.last_fullpass_impl() == 2
    traffic_full, digest_full = _traffic_for([os.path.join(ROOT, "paper_2403_18766_gb300", "csrc", f)
                                              for f in (("bm_tcx.cu", "bm_tcgen05.cuh", "bm_device.cuh")
                                                        if tensor_full else ("bm_fullpass.cu", "bm_device.cuh"))])
    roof_full = {"bound": "hbm", "achieved": full_gbs, "peak": hbm_peak, "unit": "GB/s",
                 "frac": full_gbs / hbm_peak,
                 "traffic": traffic_full.get("dram_bytes_per_launch") if traffic_full else None,
                 "source_digest": digest_full,
                 "kernel": ("tcx_fullpass_kernel<16> (tcgen05 split-TF32, certified, labels + f(C, X))"
                            if tensor_full else "fullpass_kernel<16> (FP32 ALU, certified, labels + f(C, X))"),
                 "algorithmic": f"m*n*4 = {bytes_full:.4g} bytes per launch (X read once)",
                 "avg_launch_us": t_full / max(n_full, 1) * 1e6, "peak_source": peak_src}

    # e2e: the same metric through the host-buffer C-ABI call, H2D and D2H inside
    e2e = None
    if rank == 0 or ws > 1:
        Xp = torch.from_numpy(X).pin_memory()
        # the same fit as the device-timed session (warm-up + timed rounds),
        # now from host memory with its copies, setup and final pass inside
        e2e_rounds = args.warmup + args.steps
        e2e_bud = native.make_budget(rounds=e2e_rounds, **BUDGET)
        e2e_vals, e2e_parts = [], []
        for i in range(3):
            t0 = time.perf_counter()
            _, _, r = native.fit_host(Xp, K_CLUSTERS, native.make_policy(**POLICY), e2e_bud, seed=77 + i,
                                      labels=True)
            dt = time.perf_counter() - t0
            e2e_vals.append(r["assign_rows"] * K_CLUSTERS / dt)
            e2e_parts.append((dt, r))
        dt_med, r_med = sorted(e2e_parts, key=lambda p: p[0])[1]
        e2e_value, e2e_ranks = statistics.median(e2e_vals), 1
        if ws > 1:                      # whole job: every rank's pts*k over the slowest rank's call
            t_e, w_e = aggregate(dt_med, r_med["assign_rows"] * K_CLUSTERS, dev)
            e2e_value, e2e_ranks = w_e / t_e, ws
        e2e = {"value": e2e_value, "unit": UNIT,
               "call_ms": dt_med * 1e3, "worker_ms": r_med["t_worker_s"] * 1e3,
               "fullpass_ms": r_med["t_fullpass_s"] * 1e3, "assign_rows": r_med["assign_rows"],
               "h2d_bytes_per_step": m * n * 4 * e2e_ranks,
               "d2h_bytes_per_step": (K_CLUSTERS * n * 4 + m * 4) * e2e_ranks,
               "step": f"one bigmeans_fit_host call ({e2e_rounds} rounds from scratch + final recheck + "
                       "labels) from pinned host memory: copies, workspace setup, K-means++ of round 0 and "
                       "the final full pass inside; median of 3 calls"
                       + (f"; on {ws} ranks each rank makes such a call, the value is their total pts*k over "
                          "the slowest rank's median call" if ws > 1 else "")}

    # the other configurations, one sub-object each (rank 0 of a 1-GPU run)
    extras, checks = {}, {"headline": {"C": C.cpu().numpy(), "labels": Y_fin.cpu().numpy(),
                                       "f": rep_fin["f_full"]}}
    if rank == 0 and ws == 1 and not args.no_extras:
        del Xd
        torch.cuda.empty_cache()
        extras["precision"], checks["precision"] = precision_bench(steps=5, warmup=3)
        torch.cuda.empty_cache()
        extras["batched"] = batched_bench(steps=5, warmup=3)
        torch.cuda.empty_cache()
        extras["serve"] = serve_bench(rate=20.0, n_jobs=40, warmup=3)
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(X, checks=checks)

    if rank == 0:
        line = {"metric": METRIC, "value": ptsk / t_job, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_job * 1e3 / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": config_dict(m, n),
                "roofline": roofline, "roofline_fullpass": roof_full,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk,
                "time_to_objective": {"target": "incumbent f(C, X) within 1e-4 (relative) of its value after "
                                                "the last round", "seconds": tto[0], "rounds": tto[1],
                                      "f_end": f_end, "trace": [[round(t, 6), f] for t, f in trace]},
                "detail": {"step_ms": step_ms, "lloyd_rows": rows, "worker_ms_per_launch":
                           t_worker / max(n_worker, 1) * 1e3,
                           "rescored_rows": rep1["rescored_rows"],
                           "reseeded": rep1["reseeded"] - rep0["reseeded"],
                           "sample_ms_per_step": (rep1["t_sample_s"] - rep0["t_sample_s"]) * 1e3 / args.steps,
                           "trace_cycles": [b - a for a, b in zip(rep0["trace_cycles"],
                                                                   rep1["trace_cycles"])],
                           "inexact_terms": rep1["inexact_terms"],
                           "f_incumbent": rep1["f_incumbent"], "f_final": rep_fin["f_full"],
                           "s_opt": rep_fin["s_opt"], "peaks": peak_src,
                           "worker_launches_per_round": 1}}
        if cpu and "err_vs_pure64" in cpu:
            line["err_vs_pure64"] = cpu["err_vs_pure64"]
        line.update(extras)
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_kernel_mode(args):
    """Kernel-level runs on the same workload for profiling (not the headline):
    --mode fullpass: bm_assign (labels + f) on all of X with the C of a short fit;
    --mode lloyd:    bm_lloyd on one 64,000-row sample (tol < 0: fixed iterations)."""
    import torch
    from paper_2403_18766_gb300 import native
    from paper_2403_18766_gb300.synthetic import workload
    name = args.workload or WORKLOAD
    X = workload(name, m=args.rows)
    Xd = torch.from_numpy(X).cuda()
    kc = args.k or K_CLUSTERS
    if args.centroids == "fit":      # centroids as a fit leaves them (close calls between split clusters)
        C, _, _ = native.fit(Xd, kc, native.make_policy(s_min=20000, s_max=60000, workers=8, passes=4),
                             native.make_budget(rounds=1), seed=3, labels=False)
    else:
        C = Xd[torch.arange(0, X.shape[0], X.shape[0] // kc)[:kc].cuda()].contiguous()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    S = Xd[:POLICY["s_max"]].contiguous()
    times, kern, resc = [], [], 0
    for i in range(args.warmup + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if args.mode == "fullpass":
            _, _, rep = native.assign(Xd, C)
        else:
            native.lloyd(S, C, 20, -1.0)
        torch.cuda.synchronize()
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
            if args.mode == "fullpass":
                kern.append(rep["t_fullpass_s"])
                resc = rep["rescored_rows"]
    out = {"mode": args.mode, "median_ms": statistics.median(times) * 1e3,
           "note": "wall time of the whole call (allocation, staging, prepass included)"}
    if kern:
        m, n = X.shape
        out.update({"kernel_median_ms": statistics.median(kern) * 1e3,
                    "kernel_GBps": m * (n * 4 + 4) / statistics.median(kern) / 1e9,
                    "impl": native.last_fullpass_impl(), "rescored_rows": resc})
    print(json.dumps(out))
    return 0


def _timed(fn, steps, warmup, flush):
    import torch
    ts, out = [], None
    for i in range(warmup + steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        out = fn()
        b.record()
        torch.cuda.synchronize()
        if i >= warmup:
            ts.append(a.elapsed_time(b) / 1e3)
    return statistics.median(ts), out


def precision_bench(steps=5, warmup=3, rows=None, slice_rows=200_000):
    """Workload 4: precision form of the full-data pass on 10^7 x 64, k = 100
    (100 Gaussians, Zipf(1.2) sizes): X packed once to BF16 (resident), then
    bm_assign_bf16 (tau = 1e-3) timed with CUDA events (L2 flushed between
    calls) against the HBM roofline; the exact FP32 pass (bm_assign) and the
    certified variant on the same C are timed beside it, with the label
    agreement and objective error against the exact pass.  Returns the
    sub-object and, for the FP64 check of the CPU leg, each form's f on the
    first `slice_rows` rows."""
    import torch
    from paper_2403_18766_gb300 import native
    from paper_2403_18766_gb300.synthetic import workload
    X = workload("gmm_10m_n64_k100z", m=rows)
    m, n = X.shape
    k = 100
    Xd = torch.from_numpy(X).cuda()
    # centroids as the pass meets them after a fit: one short Big-means fit
    C, _, _ = native.fit(Xd, k, native.make_policy(s_min=20000, s_max=60000, workers=8, passes=4),
                         native.make_budget(rounds=1), seed=3, labels=False)
    P = native.PackedBF16(Xd)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    clocks = ClockSampler(0)
    clocks.begin()
    t_bf, (Yb, fb, rb) = _timed(lambda: native.assign_bf16(P, C, tau=1e-3), steps, warmup, flush)
    t_tc0, _ = _timed(lambda: native.assign_bf16(P, C, tau=0.0), steps, warmup, flush)
    t_ex, (Ye, fe, re_) = _timed(lambda: native.assign(Xd, C), steps, warmup, flush)
    t_ce, (Yc, fc, rc) = _timed(lambda: native.assign_bf16(P, C, tau=1e-3, certified=True), steps, warmup, flush)
    # the fit entry point in both modes, X packed once beside its FP32 master:
    # the wall time of each call and the gap of the fast mode's f(C_best, X)
    pol_f = native.make_policy(s_min=20000, s_max=60000, workers=8, passes=4)
    bud_f = native.make_budget(rounds=1)
    t_fx, (_, _, r_fx) = _timed(lambda: native.fit_dt(Xd, k, pol_f, bud_f, seed=3, mode=native.BM_MODE_EXACT),
                                3, 1, flush)
    t_ff, (_, _, r_ff) = _timed(lambda: native.fit_dt(P, k, pol_f, bud_f, seed=3, mode=native.BM_MODE_FAST),
                                3, 1, flush)
    gap = abs(r_ff["f_full"] - r_fx["f_full"]) / r_fx["f_full"]
    fit_modes = {"exact_ms": t_fx * 1e3, "fast_ms": t_ff * 1e3, "f_exact": r_fx["f_full"],
                 "f_fast": r_ff["f_full"], "f_rel_gap": gap, "within_1e-4": bool(gap <= 1e-4),
                 "what": "bigmeans_fit_dt (W = 8, p = 4, T = 1, s in [20000, 60000]) in exact mode on the FP32 X "
                         "and in fast mode on the packed X: labels and f(C_best, X) from the exact pass or from "
                         "the precision pass (tau = 1e-3); the fit itself is the same"}
    clocks.end()
    clk = clocks.stop()
    # the same forms on the first rows, for the comparison with the FP64 oracle
    ns = min(slice_rows, m)
    Xs = Xd[:ns].contiguous()
    Ps = native.PackedBF16(Xs)
    fs = {"bf16_tau1e-3": native.assign_bf16(Ps, C, tau=1e-3)[1],
          "bf16_certified": native.assign_bf16(Ps, C, tau=1e-3, certified=True)[1],
          "exact_fp32": native.assign(Xs, C)[1]}
    check = {"X": X[:ns].copy(), "C": C.cpu().numpy(), "f": fs}
    peaks, src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    bytes_bf = m * (128 + 4 + 4)                 # packed row + norm + label
    # DRAM traffic of the call from the committed capture (per row of the
    # pass, per re-scored row of the re-score kernel), while the sources match
    tr, digest_tc = _traffic_for([os.path.join(ROOT, "paper_2403_18766_gb300", "csrc", f)
                                  for f in ("bm_tc.cu", "bm_tcgen05.cuh", "bm_device.cuh")])
    traffic_bf = (tr["dram_bytes_per_row"] * m + tr["dram_bytes_per_rescored_row"] * rb["rescored_rows"]
                  if tr and "dram_bytes_per_row" in tr else None)
    line = {"metric": "precision-form full pass (labels + f)", "value": bytes_bf / t_bf / 1e9,
            "unit": "GB/s", "higher_is_better": True, "steps": steps, "warmup": warmup,
            "config": {"workload": f"gmm_10m_n64_k100z: m={m}, n=64, 100 Gaussians (Zipf 1.2), k=100",
                       "dtype": "bf16 distance tiles, FP32 accumulate (tcgen05), FP32 re-score",
                       "tau": 1e-3, "l2": "flushed between calls"},
            "roofline": {"bound": "hbm", "achieved": bytes_bf / t_bf / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": bytes_bf / t_bf / 1e9 / hbm, "traffic": traffic_bf,
                         "source_digest": digest_tc,
                         "kernel": "tc_fullpass_kernel + rescore_kernel (tcgen05.mma kind::f16, 1-D bulk tiles)",
                         "algorithmic": "136 bytes per row (128 B packed row, 4 B norm, 4 B label)",
                         "peak_source": src},
            "ms_per_call": t_bf * 1e3, "exact_fp32_ms_per_call": t_ex * 1e3,
            "tau0_ms_per_call": t_tc0 * 1e3, "tau0_GBps": bytes_bf / t_tc0 / 1e9,
            "speedup_vs_exact_pass": t_ex / t_bf,
            "exact_kernel_ms": re_["t_fullpass_s"] * 1e3,
            "exact_kernel_GBps": m * (n * 4 + 4) / re_["t_fullpass_s"] / 1e9,
            "exact_rescored_rows": re_["rescored_rows"],
            "rescored_rows": rb["rescored_rows"],
            "label_mismatch_vs_exact": int((Yb != Ye).sum().item()),
            "f_rel_err_vs_exact": abs(fb - fe) / fe, "f_precision": fb, "f_exact": fe,
            "certified": {"ms_per_call": t_ce * 1e3, "speedup_vs_exact_pass": t_ex / t_ce,
                          "rescored_rows": rc["rescored_rows"],
                          "label_mismatch_vs_exact": int((Yc != Ye).sum().item()),
                          "f_rel_err_vs_exact": abs(fc - fe) / fe},
            "fit_modes": fit_modes,
            "clocks": clk}
    del P, Ps, Xd, Xs
    torch.cuda.empty_cache()
    return line, check


def run_precision(args):
    line, _ = precision_bench(args.steps, args.warmup, args.rows)
    print(json.dumps(line))
    return 0


def batched_bench(steps=5, warmup=3, rows=None):
    """Workload 3: 64 competing workers on one 4e6 x 32 mixture (50 Gaussians
    + 1% outliers), sample sizes octave-uniform (the integer stand-in for
    log-uniform) in [2000, 131072], k in {10, 25, 50} per worker.  Workers
    with different k cannot compete on one objective, so they form three
    Big-means groups (22 / 21 / 21 workers, k assigned round-robin), each its
    own fit; every round of all three fits is one worker launch
    (bm_fit_rounds_batch).  The cluster tile of the one-cluster-per-worker
    plan is autotuned, then timed against the worker-group plan; the faster
    runs the timed steps.  A step is one round of all 64 workers; the value
    is Lloyd pts*k/s over all groups, device-resident X, L2 flushed between
    steps."""
    import torch
    from paper_2403_18766_gb300 import native
    from paper_2403_18766_gb300.synthetic import workload
    X = workload("gmm_4m_n32_k50o", m=rows)
    m, n = X.shape
    Xd = torch.from_numpy(X).cuda()
    groups = [(10, 22), (25, 21), (50, 21)]
    pols = {k: native.make_policy(s_min=2000, s_max=131072, workers=w, passes=10, kind=1) for k, w in groups}
    native.set_worker_groups(0)
    try:
        tuned, tune_ms = native.autotune_rows_per_cta(Xd, 25, pols[25], native.make_budget(rounds=2), seed=5,
                                                      candidates=(1024, 2048, 4096, 8192))
    finally:
        native.set_worker_groups(1)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def sessions(rounds):
        return [native.FitSession(Xd, k, pols[k], native.make_budget(rounds=rounds), seed=300 + k)
                for k, _ in groups]

    def one_round(sess):
        native.rounds_batch(sess, 1)

    # plan choice: two rounds each (the second one timed)
    plan_ms = {}
    for on in (1, 0):
        native.set_worker_groups(on)
        sess = sessions(2)
        one_round(sess)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one_round(sess)
        torch.cuda.synchronize()
        plan_ms["groups" if on else f"tile_{tuned}"] = (time.perf_counter() - t0) * 1e3
        for s_ in sess:
            s_.close()
    use_groups = plan_ms["groups"] <= plan_ms[f"tile_{tuned}"]
    native.set_worker_groups(1 if use_groups else 0)
    sess = sessions(warmup + steps)
    try:
        for _ in range(warmup):
            one_round(sess)
        rep0 = [s_.report() for s_ in sess]
        clocks = ClockSampler(0)
        step_ms = []
        clocks.begin()
        for _ in range(steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            one_round(sess)
            b.record()
            torch.cuda.synchronize()
            step_ms.append(a.elapsed_time(b))
        clocks.end()
        clk = clocks.stop()
        rep1 = [s_.report() for s_ in sess]
        fin = {}
        for s_, (k, _) in zip(sess, groups):
            C, _, r = s_.finish(labels=False)
            fin[str(k)] = {"f_full": r["f_full"], "s_opt": r["s_opt"]}
    finally:
        for s_ in sess:
            s_.close()
        native.set_worker_groups(1)
        native.set_rows_per_cta(0)
    ptsk = sum((r1["assign_rows"] - r0["assign_rows"]) * k for r0, r1, (k, _) in zip(rep0, rep1, groups))
    flops = sum(2.0 * n * k * (r1["assign_rows"] - r0["assign_rows"]) for r0, r1, (k, _) in zip(rep0, rep1, groups))
    t = sum(step_ms) / 1e3
    peaks, src = _peaks()
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", NOMINAL_MAX_MHZ))
    alu_peak = sm_count * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
    tr, digest = _traffic_for([os.path.join(ROOT, "paper_2403_18766_gb300", "csrc", f)
                               for f in ("bm_worker_impl.cuh", "bm_worker.cuh", "bm_device.cuh")], "gmm_4m_n32_k50o")
    return {"metric": "Lloyd pts·k/s (batched workers, workload 3)", "value": ptsk / t, "unit": UNIT,
            "higher_is_better": True, "steps": steps, "warmup": warmup,
            "ms_per_step": t * 1e3 / steps, "dtype": "f32", "data": "synthetic",
            "roofline": {"bound": "alu", "achieved": flops / t / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": flops / t / 1e12 / alu_peak,
                         "traffic": tr.get("dram_bytes_per_launch") if tr else None, "source_digest": digest,
                         "kernel": "worker_kernel<32> (one launch for the 64 workers of the 3 fits) + "
                                   "sample_kernel<32> x 3 per step, CUDA events around the step",
                         "peak_source": f"{sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {max_mhz:.0f} MHz"},
            "plan": {"chosen": "groups" if use_groups else f"tile_{tuned}", "second_round_ms": plan_ms,
                     "autotune_round_ms": tune_ms, "tuned_rows_per_cta": tuned,
                     "worker_launches_per_step": 1},
            "groups": fin, "clocks": clk,
            "config": {"workload": f"gmm_4m_n32_k50o: m={m}, n={n}, 50 Gaussians + 1% outliers; 64 workers "
                                   "as 3 fits k=10/25/50 (22/21/21), s octave-uniform in [2000, 131072], p=10, "
                                   "all in one worker launch per round",
                       "l2": "flushed between timed steps", "step": "one round of all 64 workers"}}


def run_batched(args):
    print(json.dumps(batched_bench(args.steps, args.warmup, args.rows)))
    return 0


SERVE_N = (8, 32, 64)        # the stream's widths (128 is beyond the library's n <= 64)
SERVE_K = (5, 10, 25, 100)


def serve_bench(rate=20.0, n_jobs=40, warmup=3, pool_size=8, seed=5005):
    """Serving (workload 5): a Poisson stream of clustering jobs on one
    serving context (continuous batching under a device-memory budget).  Job
    shapes follow the stream: m log-uniform in [1e5, 2e7], n in SERVE_N, k in
    {5, 10, 25, 100}, a mixture of 2k Gaussians with 0.5% outliers, FP32 or
    BF16 storage (half of the jobs), W = 16 workers, T = 3 rounds, p = 10,
    s in [1000, min(64000, m)].  Jobs draw their data from a pool of
    `pool_size` data sets of such shapes, generated on the device before the
    clock starts and kept in pinned host memory; a job's latency runs from its
    arrival (submit) to its result on the host (H2D copy, Algorithm 1, the
    full-data pass -- BF16 for BF16 jobs -- and the D2H copy included);
    `without_h2d` gives the same less each job's copy of X to the device."""
    import torch
    from paper_2403_18766_gb300 import native
    from paper_2403_18766_gb300.synthetic import gaussian_mixture_device
    g = np.random.default_rng(seed)
    pool = []
    for i in range(pool_size):
        m = int(round(10 ** g.uniform(5.0, np.log10(2e7))))
        n = int(g.choice(SERVE_N))
        k = int(g.choice(SERVE_K))
        Xh = gaussian_mixture_device(m, n, 2 * k, seed=700 + i, outliers=0.005).cpu().pin_memory()
        pool.append((Xh, k))
    torch.cuda.synchronize()
    gaps = g.exponential(1.0 / rate, n_jobs)
    arrivals = np.cumsum(gaps) - gaps[0]
    jobs = []
    for i in range(n_jobs):
        Xh, k = pool[int(g.integers(len(pool)))]
        m = Xh.shape[0]
        pol = native.make_policy(s_min=max(1000, 2 * k), s_max=min(64000, m), workers=16, passes=10)
        jobs.append((Xh, k, pol, native.make_budget(rounds=3), 9000 + i, bool(g.integers(2))))
    free, total = torch.cuda.mem_get_info()
    budget = int(min(free * 0.6, 120 << 30))
    ctx = native.ServeContext(budget, 4)
    for Xh, k, pol, bud, sd, bf in jobs[:warmup]:          # warm-up jobs (not timed)
        ctx.wait(ctx.submit(Xh, k, pol, bud, sd, bf16=bf))
    clocks = ClockSampler(0)
    clocks.begin()
    t0 = time.perf_counter()
    ids = []
    for (Xh, k, pol, bud, sd, bf), at in zip(jobs, arrivals):
        dt = at - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        ids.append(ctx.submit(Xh, k, pol, bud, sd, bf16=bf))
    res = [ctx.wait(j) for j in ids]
    t_end = time.perf_counter() - t0
    clocks.end()
    clk = clocks.stop()
    st = ctx.stats()
    ctx.close()
    lat = np.array([r["t_done_s"] - r["t_submit_s"] for r in res])
    lat_nocopy = np.array([r["t_done_s"] - r["t_submit_s"] - r["report"]["t_h2d_s"] for r in res])
    qwait = np.array([r["t_admit_s"] - r["t_submit_s"] for r in res])
    ok = all(r["status"] == native.BM_OK for r in res)
    errors = sorted({r.get("error", "") for r in res if r["status"] != native.BM_OK})
    ptsk = sum(r["report"]["assign_rows"] * jobs[i][1] for i, r in enumerate(res))
    shapes = sorted({(int(p[0].shape[0]), int(p[0].shape[1]), p[1]) for p in pool})
    return {"metric": "p50/p99 job latency (serving, continuous batching)",
            "value": float(np.percentile(lat, 99)) * 1e3, "unit": "ms (p99)", "higher_is_better": False,
            "p50_ms": float(np.percentile(lat, 50)) * 1e3, "p99_ms": float(np.percentile(lat, 99)) * 1e3,
            "without_h2d": {"p50_ms": float(np.percentile(lat_nocopy, 50)) * 1e3,
                            "p99_ms": float(np.percentile(lat_nocopy, 99)) * 1e3,
                            "what": "the same latencies less each job's copy of X to the device (CUDA events)"},
            "queue_wait_p50_ms": float(np.percentile(qwait, 50)) * 1e3,
            "jobs": n_jobs, "bf16_jobs": int(sum(j[5] for j in jobs)), "all_ok": ok, "errors": errors[:3],
            "makespan_s": t_end, "jobs_per_s": n_jobs / t_end,
            "lloyd_ptsk_per_s": ptsk / t_end, "arrival_rate_per_s": rate,
            "peak_active": st["peak_active"], "peak_in_use_gb": st["peak_in_use_bytes"] / 1e9,
            "budget_gb": budget / 1e9, "clocks": clk, "pool_shapes_m_n_k": shapes,
            "config": {"workload": f"Poisson({rate:g}/s) jobs; m log-uniform in [1e5, 2e7], n in {list(SERVE_N)}, "
                                   "k in {5, 10, 25, 100}, 2k Gaussians + 0.5% outliers, FP32 or BF16 storage; "
                                   "W=16, p=10, T=3 rounds, s in [max(1000, 2k), min(64000, m)]",
                       "max_active": 4, "data": f"synthetic, {pool_size} data sets in pinned host memory"}}


def run_serve(args):
    line = serve_bench(rate=args.rate, n_jobs=max(8, args.steps * 2), warmup=args.warmup)
    print(json.dumps(line))
    return 0 if line["all_ok"] else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rate", type=float, default=20.0, help="serve mode: job arrivals per second")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only (no precision / batched / serve sub-objects)")
    ap.add_argument("--big-clusters", type=int, default=None, choices=[0, 1],
                    help="512-thread CTAs for the workers whose cluster is at the size cap")
    ap.add_argument("--workload", default=None, help="kernel modes: workload name (default: the headline's)")
    ap.add_argument("--rows", type=int, default=None, help="kernel modes: rows of the workload to use")
    ap.add_argument("--k", type=int, default=None, help="kernel modes: number of centroids")
    ap.add_argument("--fullpass-impl", type=int, default=0, choices=[0, 1, 2],
                    help="full-data pass: 0 by shape, 1 FP32 ALU, 2 tensor cores where they apply")
    ap.add_argument("--centroids", choices=["rows", "fit"], default="rows",
                    help="kernel modes: centroids from evenly spaced rows, or from a short fit")
    ap.add_argument("--mode", choices=["fit", "fullpass", "lloyd", "precision", "serve", "batched"], default="fit",
                    help="fit: the headline benchmark; fullpass / lloyd: one kernel family, "
                         "for profiling")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.big_clusters is not None and args.impl == "ours":
        from paper_2403_18766_gb300 import native
        native.set_big_clusters(args.big_clusters)
    if args.fullpass_impl and args.impl == "ours":
        from paper_2403_18766_gb300 import native
        native.set_fullpass_impl(args.fullpass_impl)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "batched":
        return run_batched(args)
    if args.mode == "precision":
        return run_precision(args)
    if args.mode != "fit":
        return run_kernel_mode(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
