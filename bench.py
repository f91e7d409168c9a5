"""Benchmark of the BO suggest step on GB300: candidates scored per second.

One step = one observation update of the surrogate (FP64 L^-1 / beta) plus
one prediction pass over every valid configuration (K* tiles, contraction,
row reduction, lambda, EI / PI / LCB, masked top-k): every row of the hot
path.  Workload (default): the 7-parameter GEMM-tiling-like space, 113,247
valid of 245,760 configurations, at n = 220 - K .. 220 observations.

  python bench.py [--steps K] [--warmup W] [--precision fp64|fp16x3|bf16x3|tf32]
                  [--config 1|2|3] [--impl ours|reference] [--gpus N]

Prints one JSON line (rank 0).  `value` is device time (CUDA events on the
session's stream) with the space's state resident in HBM and L2 flushed
between steps; `e2e` goes through the C ABI (bo_observe + bo_suggest: the
observation in, the pass result out) timed on the host.  Under torchrun each
rank runs an independent replica (the path has no exchange step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing
import os
import statistics
import subprocess
import sys
import tempfile
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "candidates scored/s per suggest & p50/p99 suggest latency vs plain FP64 form"
CONFIGS = {
    1: dict(name="blocks-4p: 4 params, 2,560 valid of 5,120", n_final=80, af="ei"),
    2: dict(name="gemm-7p: 7 params, 113,247 valid of 245,760", n_final=220, af="ei"),
    3: dict(name="gemm-9p: 9 params, 1,032,469 valid of 3,932,160", n_final=512, af="ei"),
}
DTYPE = {"fp64": "f64", "fp16x3": "f16x3 (fp32 accumulate)", "bf16x3": "bf16x3 (fp32 accumulate)",
         "tf32": "tf32 (fp32 accumulate)", "tf32x3": "tf32x3 (fp32 accumulate)"}
# FP64 peak if no device measurement is available: the nominal GB300 figure
FP64_NOMINAL_TFLOPS = 1.25
# Max errors against the FP64 oracle on the 10k-candidate subsample of the
# full-size states (tests/test_gpu_tc.py::test_full_size, GB300): scaled =
# |err| / max(|ref|, 1), strict = |err| / max(|ref|, 1e-3); the 1e-3 bar is
# met on sigma by FP16X3 and TF32X3 only.
PARITY = {
    (2, "fp16x3"): dict(mu=6.3e-4, sigma=9.4e-5, mu_strict=0.12, sigma_strict=1.0e-2),
    (3, "fp16x3"): dict(mu=2.4e-4, sigma=7.1e-5, mu_strict=0.067, sigma_strict=1.0e-2),
    (2, "tf32x3"): dict(mu=5.4e-4, sigma=3.4e-4, mu_strict=0.098, sigma_strict=0.34),
    (3, "tf32x3"): dict(mu=2.2e-4, sigma=1.3e-4, mu_strict=0.056, sigma_strict=1.0e-2),
    (2, "bf16x3"): dict(mu=6.3e-4, sigma=6.8e-3, mu_strict=0.12, sigma_strict=6.8),
    (3, "bf16x3"): dict(mu=2.4e-4, sigma=3.4e-3, mu_strict=0.067, sigma_strict=3.4),
    (2, "tf32"): dict(mu=5.4e-4, sigma=8.9e-2, mu_strict=0.098, sigma_strict=1.0),
    (3, "tf32"): dict(mu=2.2e-4, sigma=4.5e-2, mu_strict=0.056, sigma_strict=1.0),
}
MEETS_BAR = ("fp16x3", "tf32x3")
LAT_WARM = 50             # warm-up suggest calls before the latency sample
# dram bytes per launch of the dominant kernel from an ncu capture, keyed by the
# sha256 of the kernel source it was taken on (null once the source changes)
TRAFFIC = {
    "predict_f64": [{"bytes_per_launch": 1228544 + 0, "src_sha": "536356e59795c5b1", "n": 220, "N": 113247,
                     "capture": "profiles/predict_f64_gemm7p_n220.md"}],
    "predict_tc_fp16x3": [
        {"bytes_per_launch": 10722048 + 3072, "src_sha": "6a86536e3304ae4b", "n": 512, "N": 1032469,
         "capture": "profiles/predict_tc_fp16x3_gemm9p_n512.md"},
        {"bytes_per_launch": 1004032 + 0, "src_sha": "6a86536e3304ae4b", "n": 220, "N": 113247,
         "capture": "profiles/predict_tc_fp16x3_gemm7p_n220.md"},
    ],
    "predict_tc_tf32x3": [
        {"bytes_per_launch": 11245568 + 1792, "src_sha": "6a86536e3304ae4b", "n": 512, "N": 1032469,
         "capture": "profiles/predict_tc_tf32x3_gemm9p_n512.md"},
    ],
}


def log(msg):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def space_for(cfg):
    from paper_2111_14991_gb300 import workloads as W
    return {1: W.config1_space, 2: W.config2_space, 3: W.config3_space}[cfg]()


def observations(sp, cfg, count, seed=0):
    from paper_2111_14991_gb300 import workloads as W
    land = W.Landscape(sp, seed)
    idx = W.clustered_observations(land, count, seed)
    y = np.array([land(i) for i in idx])
    return idx, y


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while active."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        sm, mx, reasons = [], None, set()
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                sm.append(float(f[1]))
                mx = float(f[2])
                for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                      "sw_power_cap"), f[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        except (OSError, ValueError):
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_sha(precision):
    src = "bo_predict_f64.cu" if precision == "fp64" else "bo_predict_tc.cu"
    path = os.path.join(ROOT, "paper_2111_14991_gb300", "csrc", src)
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def flops_per_candidate(n, d):
    """Algorithmic flops of one candidate: the triangular contraction n(n+1),
    the row reductions 4n, and the Matern cross-covariance n(3d + 12)."""
    return n * (n + 1) + 4 * n + n * (3 * d + 12)


def aggregate(units, seconds, world, device="cpu"):
    """Whole-job throughput of independent replicas: the units every rank
    processed over the slowest rank's time (max over ranks)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(units), float(seconds)], dtype=torch.float64, device=device)
        tot = t[:1].clone()
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        mx = t[1:].clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        units, seconds = float(tot.item()), float(mx.item())
    return units / seconds, seconds


def kernel_only(args):
    """Build the final-state session and launch the prediction kernel a few
    times (the command the ncu captures profile)."""
    import torch
    from paper_2111_14991_gb300 import Space, build
    build.build()
    cfg = CONFIGS[args.config]
    sp = space_for(args.config)
    idx, y = observations(sp, args.config, cfg["n_final"], seed=0)
    s = Space(sp.grids, sp.invalid, precision=args.precision, n_max=max(cfg["n_final"], 32))
    for i, v in zip(idx, y):
        s.observe(int(i), float(v))
    s.sync()
    st = torch.cuda.current_stream()
    ts = []
    for _ in range(args.kernel_only):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        s.predict_enqueue()
        e1.record(st)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    s.close()
    print(json.dumps({"kernel_only": args.kernel_only, "config": cfg["name"], "precision": args.precision,
                      "n": cfg["n_final"], "ms": ts}))


def tc_mma_flops(n, N, precision):
    """Tensor-core flops the kernel issues: 3 products (1 for TF32), chunks of
    32 observations (16 for the TF32 forms), each chunk's N range running from
    its first row to n_pad."""
    cw = 16 if precision in ("tf32", "tf32x3") else 32
    n_pad = (n + 31) // 32 * 32
    cols = sum(n_pad - c * cw for c in range(n_pad // cw))
    return (1 if precision == "tf32" else 3) * 2 * 128 * cw * cols * ((N + 127) // 128)


def traffic_for(key, precision, n, N):
    """Per-launch DRAM bytes from the committed ncu capture of this kernel source
    and launch size, else None."""
    for tr in TRAFFIC.get(key, []):
        if tr["src_sha"] == kernel_sha(precision) and tr["n"] == n and tr["N"] == N:
            return tr["bytes_per_launch"]
    return None


ALU = {}          # measured arithmetic peaks of this device (filled once per run)


def measure_alu():
    """The FP64 / FP32 / f32x2 FMA and MUFU issue rates of this GPU (the
    library's probe kernels), and torch's float64 matmul (cuBLAS DGEMM) beside."""
    import torch
    from paper_2111_14991_gb300 import bo
    r = bo.measure_alu_peaks()
    a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    b = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = 1e30
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    r["dgemm_tflops"] = 2.0 * 4096 ** 3 / best / 1e12
    del a, b
    ALU.update({k: round(v, 3) if isinstance(v, float) else v for k, v in r.items()})
    return ALU


def kstar_roofline(precision, n, d, N, k1_time):
    """Second roofline of the tensor-core pass: the K* producers' FP32 work,
    (3d + 12) flops and 2 MUFU operations per (candidate, observation) pair,
    against the measured packed-FP32 and MUFU rates."""
    pairs = float(N) * n
    fl = pairs * (3 * d + 12) / k1_time / 1e12
    mu = pairs * 2 / k1_time / 1e9
    out = {"bound": "alu", "what": "K* producers: (3d+12) FP32 flops + 2 MUFU per pair", "pairs": pairs,
           "achieved_tflops": round(fl, 2), "achieved_mufu_gops": round(mu, 1)}
    if ALU:
        out.update(peak_tflops=ALU["fp32x2_fma_tflops"], frac=round(fl / ALU["fp32x2_fma_tflops"], 4),
                   peak_mufu_gops=ALU["mufu_gops"], mufu_frac=round(mu / ALU["mufu_gops"], 4),
                   peak_source="measured on this GPU (bo_measure_alu_peaks: f32x2 FMA, ex2 + rsqrt)")
    return out


def roofline_for(precision, n, d, N, k1_time):
    alg = float(N) * n * (n + 1)                       # triangular contraction, flops
    if precision == "fp64":
        fl = float(flops_per_candidate(n, d)) * N
        ach = fl / k1_time / 1e12
        peak = ALU.get("fp64_fma_tflops", FP64_NOMINAL_TFLOPS)
        return {"bound": "alu", "kernel": "predict_f64_kernel", "achieved": round(ach, 4),
                "peak": peak, "unit": "TFLOP/s", "frac": round(ach / peak, 4),
                "peak_source": ("measured on this GPU: DFMA probe (bo_measure_alu_peaks); cuBLAS DGEMM "
                                f"{ALU['dgemm_tflops']} TFLOP/s beside" if ALU else
                                "nominal GB300 FP64 (no device measurement)"),
                "traffic": traffic_for("predict_f64", precision, n, N),
                "flops_per_launch": fl, "launch_s": k1_time}
    peaks = _peaks()
    tf = precision in ("tf32", "tf32x3")
    peak = peaks["bf16_tflops"] * (0.5 if tf else 1.0)
    ach = alg / k1_time / 1e12
    issued = tc_mma_flops(n, N, precision) / k1_time / 1e12
    return {"bound": "tensor", "kernel": "predict_tc_kernel<%s>" % precision, "achieved": round(ach, 2),
            "peak": peak, "unit": "TFLOP/s", "frac": round(ach / peak, 4),
            "peak_source": ("measured bf16 burst (MEASURED_PEAKS.json)" + (" x 1/2 nominal tf32 ratio"
                            if tf else "; f16 runs at the bf16 rate")),
            "mma_issued_tflops": round(issued, 1), "mma_issued_frac": round(issued / peak, 4),
            "traffic": traffic_for("predict_tc_" + precision, precision, n, N),
            "flops_per_launch": alg, "launch_s": k1_time,
            "kstar": kstar_roofline(precision, n, d, N, k1_time)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {"bf16_tflops": 1900.0, "hbm_gbs": 6800.0, "fallback": True}


def measure_device(cfg_id, precision, steps, warm, flush, stream):
    """Device-resident steps (observe + predict + acquire), CUDA events on the
    session's stream, L2 flushed between steps; then the prediction kernel alone."""
    import torch
    from paper_2111_14991_gb300 import Space
    cfg = CONFIGS[cfg_id]
    sp = space_for(cfg_id)
    n_final = cfg["n_final"]
    idx, y = observations(sp, cfg_id, n_final, seed=0)
    n0 = max(2, n_final - steps - warm)
    s = Space(sp.grids, sp.invalid, af=cfg["af"], precision=precision, n_max=max(n_final, 32))
    for i, v in zip(idx[:n0], y[:n0]):
        s.observe(int(i), float(v))
    s.sync()
    tune = s.autotune(reps=3) if precision != "fp64" else None
    times, scored, launches = [], 0, 0
    for t in range(warm + steps):
        j = n0 + t
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = s.launch_count()
        e0.record(stream)
        s.replay_enqueue([idx[j]], [y[j]])
        e1.record(stream)
        r = s.replay_fetch(1)[0]
        if t >= warm:
            times.append(e0.elapsed_time(e1) / 1e3)
            scored += r["n_scored"]
            launches += s.launch_count() - l0
    k1 = []
    for _ in range(max(3, min(10, steps))):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.predict_enqueue()
        e1.record(stream)
        torch.cuda.synchronize()
        k1.append(e0.elapsed_time(e1) / 1e3)
    s.close()
    n_last = n0 + warm + steps
    return dict(sp=sp, idx=idx, y=y, n0=n0, n_last=n_last, times=times, scored=scored, launches=launches,
                k1=statistics.median(k1), value=scored / sum(times), tune=tune)


def _session_inputs(job):
    """One session of the batched / served configuration: its space, observation
    trace and landscape values (runs in a spawned worker process, no CUDA)."""
    seed, s, spec, kind, extra = job
    from paper_2111_14991_gb300 import workloads as W
    sp = W.batched_space(seed, s, spec)
    land = W.Landscape(sp, s)
    out = dict(grids=sp.grids, invalid=sp.invalid, n_valid=sp.n_valid, d=sp.d, n_obs=spec[2])
    if kind == "batched":
        idx = W.clustered_observations(land, spec[2], s)
        out.update(idx=idx, y=land.clean(idx))
    else:
        init = W.clustered_observations(land, min(spec[2], 512 - extra - 8), s)
        rng = np.random.default_rng(seed * 1000003 + s + 99)
        rest = np.setdiff1d(rng.choice(sp.n_valid, min(sp.n_valid, len(init) + extra), replace=False), init)
        rng.shuffle(rest)
        out.update(idx=init, y=land.clean(init), rest=rest, y_rest=land.clean(rest))
    return out


def session_inputs(count, kind, seed=0, extra=160):
    """Sessions of the batched configuration (d ~ U{3..9}, N ~ log-U[1k, 500k],
    n ~ U{20..400}), built by a pool of spawned host processes."""
    from paper_2111_14991_gb300 import workloads as W
    specs = W.batched_specs(count, seed=seed)
    jobs = [(seed, s, specs[s], kind, extra) for s in range(count)]
    workers = max(1, min(16, os.cpu_count() or 1))
    with ProcessPoolExecutor(max_workers=workers, mp_context=multiprocessing.get_context("spawn")) as ex:
        return list(ex.map(_session_inputs, jobs, chunksize=2))


def batched_workload(count, steps, warm, precision, seed=0):
    """Sessions of the batched configuration; the last warm + steps
    observations of each session are held back for the timed steps."""
    from paper_2111_14991_gb300 import Batch, Space
    sess = session_inputs(count, "batched", seed=seed)
    spaces = []
    n_max = min(512, max(x["n_obs"] for x in sess) + 1)
    for x in sess:
        spaces.append(Space(x["grids"], x["invalid"], precision=precision, af="ei", n_max=n_max))
    batch = Batch(spaces)
    hold = warm + steps
    rounds = max(len(x["idx"]) for x in sess) - hold
    for r in range(rounds):                      # initial observations, one batched update per round
        ii = [int(x["idx"][r]) if r < len(x["idx"]) - hold else -1 for x in sess]
        yy = [float(x["y"][r]) if r < len(x["idx"]) - hold else 0.0 for x in sess]
        batch.observe(ii, yy)
    return sess, spaces, batch


def measure_batched(count, steps, warm, precision, stream):
    """Device-timed batched steps: one observation per session (batched update)
    and one prediction pass per session (one persistent launch)."""
    import torch
    sess, spaces, batch = batched_workload(count, steps, warm, precision)
    hold = warm + steps
    times, scored, flops, tune = [], 0, 0.0, None
    tune_flops = 0.0
    for t in range(warm + steps):
        if t == warm:
            # pipeline shapes of the batched launch, timed on the previous pass's state
            # (its median kernel time is the batched prediction kernel alone)
            tune = batch.autotune(reps=3)
            n_prev = [len(x["idx"]) - hold + t for x in sess]
            tune_flops = sum(float(x["n_valid"]) * n * (n + 1) for x, n in zip(sess, n_prev))
        ii = [int(x["idx"][len(x["idx"]) - hold + t]) for x in sess]
        yy = [float(x["y"][len(x["y"]) - hold + t]) for x in sess]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = batch.launch_count()
        e0.record(stream)
        st = batch.observe(ii, yy)
        idx, st2, info = batch.suggest()
        e1.record(stream)
        torch.cuda.synchronize()
        assert not st.any() and not st2.any(), (st, st2)
        if t >= warm:
            times.append(e0.elapsed_time(e1) / 1e3)
            scored += sum(x["n_scored"] for x in info)
            n_now = [len(x["idx"]) - hold + t + 1 for x in sess]
            flops += sum(float(x["n_valid"]) * n * (n + 1) for x, n in zip(sess, n_now))
    launches = batch.launch_count()
    batch.close()
    for sp in spaces:
        sp.close()
    return dict(value=scored / sum(times), times=times, flops=flops, sessions=count,
                candidates=sum(x["n_valid"] for x in sess), launches=launches, tune=tune,
                tune_flops=tune_flops)


def measure_serving(count, rate, duration, precision, extra=160, seed=0, budget_gb=120):
    """Open-loop serving: Poisson arrivals at `rate` requests/s (observe one new
    point + suggest) spread uniformly over `count` live sessions of the batched
    configuration's sizes, for `duration` seconds; then a closed-loop run with
    one request of every session always in flight (saturation)."""
    from paper_2111_14991_gb300 import Server
    t_gen = time.time()
    sess = session_inputs(count, "served", seed=seed, extra=extra)
    t_gen = time.time() - t_gen
    log(f"served: {count} sessions generated in {t_gen:.1f} s")
    srv = Server(budget_bytes=budget_gb << 30, max_sessions=count)
    rng = np.random.default_rng(seed + 99)
    sids, pending = [], []
    t_setup = time.time()
    for x in sess:                               # every session opened (admitted) before any request
        sids.append(srv.open(x["grids"], x["invalid"], precision=precision, af="ei", n_max=512))
        pending.append(list(zip(x["rest"].tolist(), x["y_rest"].tolist())))
    # tags: initial observations WARM + k, open loop k, closed loop CLOSED + session
    WARM, CLOSED = 1 << 40, 1 << 41
    n_warm = 0
    for sid, x in zip(sids, sess):
        for i, v in zip(x["idx"], x["y"]):
            srv.submit(sid, int(i), float(v), tag=WARM + n_warm, suggest=False)
            n_warm += 1
    t_end = time.time() + 300
    errors, got = 0, 0
    while got < n_warm and time.time() < t_end:
        cs = srv.poll(1 << 14, wait_ms=20)
        got += len(cs)
        errors += sum(c["status"] != 0 for c in cs)
    t_setup = time.time() - t_setup
    st = srv.stats()
    log(f"served: initial observations {got}/{n_warm} in {t_setup:.1f} s, "
        f"{st['iterations']} iterations, {errors} errors")
    if got < n_warm:
        srv.close()
        return {"sessions": count, "error": f"initial observations incomplete after {t_setup:.0f} s"}
    sid_pos = {sid: k for k, sid in enumerate(sids)}
    # ---- open loop
    n_req = int(rate * duration)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    who = rng.integers(0, count, size=n_req)
    done, submitted = [], 0
    t0 = srv.now()
    for k in range(n_req):
        while srv.now() - t0 < arrivals[k]:
            done += srv.poll(4096, wait_ms=0)
        s = int(who[k])
        if pending[s]:
            i, v = pending[s].pop()
            srv.submit(sids[s], i, v, tag=k)
            submitted += 1
    t_end = time.time() + 120
    while len(done) < submitted and time.time() < t_end:
        done += srv.poll(4096, wait_ms=20)
    assert all(c["tag"] < WARM for c in done)
    log(f"served: open loop {len(done)}/{submitted} completed")
    lat = np.array([c["t_done"] - c["t_submit"] for c in done if c["idx"] >= 0])
    span = max(c["t_done"] for c in done) - t0
    scored = sum(c["info"]["n_scored"] for c in done if c["idx"] >= 0)
    open_loop = {"requests": len(lat), "errors": sum(c["status"] != 0 for c in done),
                 "rate_req_s": rate, "duration_s": round(span, 3),
                 "p50_ms": round(1e3 * float(np.percentile(lat, 50)), 3),
                 "p99_ms": round(1e3 * float(np.percentile(lat, 99)), 3),
                 "candidates_per_s": round(scored / span, 1)}
    # ---- closed loop: every session keeps one request in flight
    it0 = srv.stats()
    t0 = srv.now()
    inflight = 0
    for s in range(count):
        if pending[s]:
            i, v = pending[s].pop()
            srv.submit(sids[s], i, v, tag=CLOSED + s)
            inflight += 1
    scored, n_done, t_stop, lat_c, errs_c = 0, 0, t0 + duration, [], 0
    while inflight > 0 and srv.now() < t_stop:
        for c in srv.poll(4096, wait_ms=5):
            assert c["tag"] >= CLOSED, c["tag"]
            inflight -= 1
            n_done += 1
            errs_c += c["status"] != 0
            scored += c["info"]["n_scored"]
            lat_c.append(c["t_done"] - c["t_submit"])
            s = sid_pos[c["session"]]
            if pending[s]:
                i, v = pending[s].pop()
                srv.submit(sids[s], i, v, tag=CLOSED + s)
                inflight += 1
    span = srv.now() - t0
    t_end = time.time() + 120
    while inflight > 0 and time.time() < t_end:
        inflight -= len(srv.poll(4096, wait_ms=20))
    st = srv.stats()
    log(f"served: closed loop {n_done} requests in {span:.1f} s")
    closed_loop = {"requests": n_done, "errors": int(errs_c), "duration_s": round(span, 3),
                   "candidates_per_s": round(scored / span, 1),
                   "iterations": st["iterations"] - it0["iterations"],
                   "p50_ms": round(1e3 * float(np.percentile(lat_c, 50)), 3) if lat_c else None,
                   "p99_ms": round(1e3 * float(np.percentile(lat_c, 99)), 3) if lat_c else None}
    stats = srv.stats()
    srv.close()
    return {"sessions": count, "budget_gb": budget_gb, "candidates": sum(x["n_valid"] for x in sess),
            "open_loop": open_loop, "closed_loop": closed_loop, "admitted": stats["admitted"],
            "bytes_in_use": stats["bytes_in_use"], "setup_s": round(t_setup, 1),
            "init_errors": int(errors)}


def measure_latency(cfg_id, precision, reps, flush):
    """bo_suggest latency (host entry to index returned) at the final state of
    a configuration, after LAT_WARM warm-up calls, L2 flushed before each call."""
    import torch
    from paper_2111_14991_gb300 import Space
    cfg = CONFIGS[cfg_id]
    sp = space_for(cfg_id)
    idx, y = observations(sp, cfg_id, cfg["n_final"], seed=0)
    s = Space(sp.grids, sp.invalid, af=cfg["af"], precision=precision, n_max=max(cfg["n_final"], 32))
    for i, v in zip(idx, y):
        s.observe(int(i), float(v))
    lat, scored = [], 0
    for t in range(LAT_WARM + reps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = s.suggest()
        if t >= LAT_WARM:
            lat.append(time.perf_counter() - t0)
            scored += info["n_scored"]
    s.close()
    return {"p50_ms": round(1e3 * float(np.percentile(lat, 50)), 4),
            "p99_ms": round(1e3 * float(np.percentile(lat, 99)), 4), "calls": len(lat),
            "candidates_per_s": round(scored / sum(lat), 1),
            "what": "bo_suggest host entry to index returned, n = %d" % cfg["n_final"]}


def run_ours(args, rank, world):
    import torch
    from paper_2111_14991_gb300 import Space, build
    build.build()
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    cfg = CONFIGS[args.config]
    steps, warm = args.steps, args.warmup
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # 256 MB > 129 MB L2
    stream = torch.cuda.current_stream()
    measure_alu()
    log(f"alu peaks {ALU}")

    with ClockSampler(dev) as clk:
        m = measure_device(args.config, args.precision, steps, warm, flush, stream)
    clocks = clk.summary()
    sp, idx, y, n0, n_last = m["sp"], m["idx"], m["y"], m["n0"], m["n_last"]
    N = sp.n_valid
    tot = sum(m["times"])

    # ---- end to end through the C ABI: observe (in) + suggest (result out), host clock
    s = Space(sp.grids, sp.invalid, af=cfg["af"], precision=args.precision, n_max=max(cfg["n_final"], 32))
    for i, v in zip(idx[:n0], y[:n0]):
        s.observe(int(i), float(v))
    for t in range(warm):
        j = n0 + t
        s.observe(int(idx[j]), float(y[j]))
        s.suggest()
    e2e_t, e2e_scored = [], 0
    for t in range(steps):
        j = n0 + warm + t
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.observe(int(idx[j]), float(y[j]))
        info = s.suggest()
        e2e_t.append(time.perf_counter() - t0)
        e2e_scored += info["n_scored"]
    # suggest latency at the final state (single AF: every call is a full pass)
    lat = []
    for t in range(LAT_WARM + max(args.latency_reps, steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.suggest()
        if t >= LAT_WARM:
            lat.append(time.perf_counter() - t0)
    s.close()
    e2e_tot = sum(e2e_t)

    # ---- the other forms on the same GPU (device-timed, same recipe)
    forms = {}
    if not args.no_forms:
        form_list = ((2, "fp64"), (2, "fp16x3"), (2, "tf32x3"), (3, "fp16x3"), (3, "tf32x3"), (3, "bf16x3"),
                     (3, "tf32"), (3, "fp64"))
        for fcfg, fprec in form_list:
            if (fcfg, fprec) == (args.config, args.precision):
                continue
            f = measure_device(fcfg, fprec, steps if fprec != "fp64" or fcfg != 3 else 3, 3, flush, stream)
            log(f"form config{fcfg}/{fprec}: {f['value']:.4g} candidates/s, kernel {1e3 * f['k1']:.3f} ms")
            form = {
                "value": round(f["value"], 1), "unit": "candidates/s",
                "ms_per_step": round(1e3 * sum(f["times"]) / len(f["times"]), 4),
                "n_obs": f"{f['n0'] + 4}..{f['n_last']}", "autotune": f["tune"],
                "roofline": roofline_for(fprec, f["n_last"], f["sp"].d, f["sp"].n_valid, f["k1"])}
            if fprec != "fp64":
                par = PARITY.get((fcfg, fprec))
                form["parity"] = dict(par or {}, bar="1e-3 scaled on mu and sigma",
                                      meets_bar=fprec in MEETS_BAR,
                                      note=None if fprec in MEETS_BAR else "does not meet 1e-3 on sigma",
                                      source="tests/test_gpu_tc.py::test_full_size, 10k-candidate subsample")
            forms[f"config{fcfg}/{fprec}"] = form
        lat1 = measure_latency(1, "fp64", args.latency_reps, flush)
        forms["config1/fp64-latency"] = dict(lat1, workload=CONFIGS[1]["name"])
        if not args.no_serving:
            forms["config5/fp16x3-served"] = measure_serving(args.serve_sessions, 2000.0, 4.0, "fp16x3")
        if not args.no_batched:
            bsteps = max(3, min(steps, 10))
            f = measure_batched(args.batch_sessions, bsteps, 3, "fp16x3", stream)
            log(f"batched: {f['value']:.4g} candidates/s")
            peak = _peaks()["bf16_tflops"]
            k_s = f["tune"]["best_ms"] / 1e3
            ach = f["tune_flops"] / k_s / 1e12
            step_ach = f["flops"] / sum(f["times"]) / 1e12
            forms["config4/fp16x3-batched"] = {
                "value": round(f["value"], 1), "unit": "candidates/s",
                "ms_per_step": round(1e3 * sum(f["times"]) / len(f["times"]), 4),
                "sessions": f["sessions"], "candidates": f["candidates"], "autotune": f["tune"],
                "what": "per step: one batched update + one batched prediction pass of every session",
                "l2": "working set > L2 (no flush)",
                "roofline": {"bound": "tensor", "kernel": "predict_tc_kernel<fp16x3> over all sessions (one "
                                                          "persistent launch)",
                             "achieved": round(ach, 2), "peak": peak, "unit": "TFLOP/s",
                             "frac": round(ach / peak, 4), "launch_s": k_s, "flops_per_launch": f["tune_flops"],
                             "peak_source": "measured bf16 burst (MEASURED_PEAKS.json); launch time = the "
                                            "autotuner's median CUDA-event time of the chosen shape",
                             "whole_step_tflops": round(step_ach, 2), "traffic": None}}

    value, tot = aggregate(m["scored"], tot, world, "cuda")
    e2e_value, e2e_tot = aggregate(e2e_scored, e2e_tot, world, "cuda")
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "candidates/s", "n_gpus": world,
        "steps": steps, "warmup": warm, "ms_per_step": round(1e3 * tot / steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.precision], "data": "synthetic (seeded landscape, clustered BO-like trace)",
        "config": {"workload": cfg["name"], "n_obs": f"{n0 + warm + 1}..{n_last}",
                   "precision": args.precision, "af_pass": "ei+poi+lcb top-3 each",
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
        "latency_ms": {"p50": round(1e3 * float(np.percentile(lat, 50)), 4),
                       "p99": round(1e3 * float(np.percentile(lat, 99)), 4), "calls": len(lat),
                       "what": "bo_suggest host entry to index returned, n = %d" % n_last},
        "e2e": {"value": round(e2e_value, 1), "unit": "candidates/s", "h2d_bytes_per_step": 16,
                "d2h_bytes_per_step": 400, "what": "bo_observe(idx, y) + bo_suggest, host clock"},
        "gpu_launches": m["launches"],
        "roofline": roofline_for(args.precision, n_last, sp.d, N, m["k1"]),
        "alu_peaks": dict(ALU),
        "clocks": clocks,
        "forms": forms,
    }
    return out


def cpu_baseline_runs(cfg_id, runs=5, run_s=2.0):
    """The oracle, as it stands, on the host: `runs` timed runs of one
    suggest's prediction + scores over 20k-candidate batches drawn from the
    valid configurations at the final state (at least run_s seconds each; the
    fit, done once, is charged pro rata)."""
    import oracle as O
    sp = space_for(cfg_id)
    cfg = CONFIGS[cfg_id]
    idx, y = observations(sp, cfg_id, cfg["n_final"], seed=0)
    coords = sp.valid_coords()
    t0 = time.perf_counter()
    fit = O.gp_fit(coords[idx], y, 1.5, 1.5, 1e-10)
    t_fit = time.perf_counter() - t0
    rng = np.random.default_rng(1)
    sample = min(sp.n_valid, 20000)
    fplus = float(np.min((y - y.mean()) / y.std()))
    rates, total = [], 0
    for _ in range(runs):
        done, t_pred = 0, 0.0
        while t_pred < run_s:
            sel = rng.choice(sp.n_valid, sample, replace=False)
            t0 = time.perf_counter()
            mu, var = O.gp_posterior(fit, coords[sel])
            sd = np.sqrt(var)
            for af in ("ei", "poi", "lcb"):
                O.masked_topk(O.acquisition(af, mu, sd, fplus, 0.1), np.ones(len(sel), bool), 3)
            t_pred += time.perf_counter() - t0
            done += sample
        rates.append(done / (t_pred + t_fit * done / sp.n_valid))
        total += done
    cores = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        cores = max(int(i.get("num_threads", 1)) for i in threadpool_info()) or cores
    except Exception:
        pass
    if os.environ.get("OPENBLAS_NUM_THREADS") == "1":
        cores = 1
    return {"value": round(statistics.median(rates), 1), "runs": [round(r, 1) for r in rates], "cores": cores,
            "sample": f"{runs} runs of >= {run_s:.0f} s, {total} candidates in batches of {sample} drawn from the "
                      f"{sp.n_valid} at n = {cfg['n_final']} (fit once, prediction + EI/PI/LCB top-3)"}


def cpu_baseline(cfg_id):
    """Median of 5 oracle runs on all host cores (numpy / OpenBLAS threads),
    and the same on one thread in a child process (BLAS limited to 1 thread)."""
    allc = cpu_baseline_runs(cfg_id)
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    single = None
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-variant", "single",
                            "--config", str(cfg_id)], env=env, capture_output=True, text=True, timeout=600)
        single = json.loads(r.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError) as e:
        single = {"error": str(e)[:200]}
    return {"value": allc["value"], "unit": "candidates/s", "cores": allc["cores"], "kind": "oracle",
            "sample": allc["sample"], "stat": "median of 5 runs", "runs": allc["runs"],
            "single_thread": dict(single, unit="candidates/s", kind="oracle", stat="median of 5 runs")}


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores, on
    the same workload, observation range and step as this build's line (one
    step = fit on the step's n observations + prediction and EI / PI / LCB
    top-3 over a bounded sample of the valid configurations)."""
    import oracle as O
    cfg = CONFIGS[args.config]
    sp = space_for(args.config)
    idx, y = observations(sp, args.config, cfg["n_final"], seed=0)
    coords = sp.valid_coords()
    per_step = min(sp.n_valid, 20000)
    rng = np.random.default_rng(2)
    n0 = max(2, cfg["n_final"] - args.steps - args.warmup)
    times = []
    for t in range(args.warmup + args.steps):
        n = n0 + t + 1
        sel = rng.choice(sp.n_valid, per_step, replace=False)
        t0 = time.perf_counter()
        yn = y[:n]
        fit = O.gp_fit(coords[idx[:n]], yn, 1.5, 1.5, 1e-10)
        mu, var = O.gp_posterior(fit, coords[sel])
        sd = np.sqrt(var)
        fplus = float(np.min((yn - yn.mean()) / yn.std()))
        for af in ("ei", "poi", "lcb"):
            O.masked_topk(O.acquisition(af, mu, sd, fplus, 0.1), np.ones(per_step, bool), 3)
        if t >= args.warmup:
            times.append(time.perf_counter() - t0)
    value = per_step * len(times) / sum(times)
    cores = os.cpu_count()
    out = {"metric": METRIC, "value": round(value, 1), "unit": "candidates/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sum(times) / len(times), 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded landscape, clustered BO-like trace)", "impl": "reference",
           "config": {"workload": cfg["name"], "n_obs": f"{n0 + args.warmup + 1}..{n0 + args.warmup + args.steps}",
                      "precision": "fp64", "af_pass": "ei+poi+lcb top-3 each",
                      "parallelism": f"replicas x{args.gpus}"},
           "cpu_baseline": {"value": round(value, 1), "unit": "candidates/s", "cores": cores, "kind": "oracle",
                            "sample": f"{per_step} of the {sp.n_valid} valid configurations per step, drawn at "
                                      "random; fit + predict + EI/PI/LCB top-3"},
           "e2e": {"value": round(value, 1), "unit": "candidates/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def tuning_quality(reps, budget=220, n_init=20):
    """Sec. IV protocol on the paper-shaped synthetic kernels: mean MAE of the
    best configuration found (evaluations 40..220) per kernel and strategy,
    and each strategy's MDF.  BO strategies run through the library with
    maximin initial sampling; random search is repeated three times as often
    (the paper repeats it more for its variance)."""
    import numpy as np
    from paper_2111_14991_gb300 import build
    from paper_2111_14991_gb300 import workloads as W
    from paper_2111_14991_gb300.loop import mae, mdf, minimize, random_search
    build.build()
    strategies = {"bo-ei-fp64": dict(af="ei", precision="fp64"),
                  "bo-ei-fp16x3": dict(af="ei", precision="fp16x3"),
                  "bo-multi-fp16x3": dict(af="multi", precision="fp16x3"),
                  "bo-advanced_multi-fp16x3": dict(af="advanced_multi", precision="fp16x3"),
                  "random": None}
    kernels = ["gemm", "conv", "pnpoly", "expdist", "adding"]
    mean_mae = {k: {} for k in strategies}
    t0 = time.time()
    for name in kernels:
        sp = W.paper_shaped_space(name)
        ok = np.ones(sp.n_valid, bool) if sp.runtime_invalid is None else ~sp.runtime_invalid
        for strat, params in strategies.items():
            errs = []
            for r in range(reps * (3 if params is None else 1)):
                land = W.Landscape(sp, 100 + r)
                f_opt = float(np.min(land.clean(np.flatnonzero(ok))))
                truth = lambda i, land=land: float(land.clean([i])[0])
                if params is None:
                    idx, val = random_search(land, sp.n_valid, budget=budget, seed=r)
                else:
                    idx, val = minimize(land, sp.grids, sp.invalid, budget=budget, n_init=n_init, seed=r,
                                        **params)
                errs.append(mae(idx, val, truth, f_opt))
            mean_mae[strat][name] = round(float(np.mean(errs)), 5)
    factors = mdf(mean_mae)
    return {"quality": "Sec. IV protocol (MAE over evaluations 40..220, MDF across kernels)",
            "data": "synthetic paper-shaped landscapes (seeded), 5% lognormal noise",
            "budget": budget, "n_init": n_init, "init": "maximin", "reps_bo": reps, "reps_random": 3 * reps,
            "mean_mae": mean_mae, "mdf": {k: [round(a, 4), round(b, 4)] for k, (a, b) in factors.items()},
            "seconds": round(time.time() - t0, 1)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", type=int, default=2, choices=sorted(CONFIGS))
    ap.add_argument("--precision", default="fp64", choices=sorted(DTYPE))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--latency-reps", type=int, default=1000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the other precision forms")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched (256-session) form")
    ap.add_argument("--batch-sessions", type=int, default=256)
    ap.add_argument("--serve-sessions", type=int, default=1024)
    ap.add_argument("--cpu-variant", default=None, choices=["single", "all"],
                    help="(internal) time the oracle baseline in this process and print it")
    ap.add_argument("--no-serving", action="store_true", help="skip the served form")
    ap.add_argument("--kernel-only", type=int, default=0,
                    help="only launch the prediction kernel this many times at the final state")
    ap.add_argument("--quality", type=int, default=0,
                    help="run the tuning-quality protocol with this many repeats per BO strategy instead")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.cpu_variant:
        print(json.dumps(cpu_baseline_runs(args.config)))
        return
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    if args.kernel_only:
        kernel_only(args)
        return
    if args.quality:
        if rank == 0:
            print(json.dumps(tuning_quality(args.quality)))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
        dist.barrier()
    out = run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.config)
            log("cpu baseline done")
        print(json.dumps(out))


if __name__ == "__main__":
    main()
