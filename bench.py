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
import os
import statistics
import subprocess
import sys
import tempfile
import time

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
         "tf32": "tf32 (fp32 accumulate)"}
# FP64 peak: the recipe's nominal GB300 figure (no measured FP64 peak exists for this machine)
FP64_PEAK_TFLOPS = 1.25
# dram bytes per launch of the dominant kernel from an ncu capture, keyed by the
# sha256 of the kernel source it was taken on (null once the source changes)
TRAFFIC = {
    "predict_f64": [{"bytes_per_launch": 1117440 + 0, "src_sha": "7db7286ecbec0617", "n": 220, "N": 113247,
                     "capture": "profiles/predict_f64_gemm7p_n220.md"}],
    "predict_tc_fp16x3": [
        {"bytes_per_launch": 10716672 + 3584, "src_sha": "881cb10161712188", "n": 512, "N": 1032469,
         "capture": "profiles/predict_tc_fp16x3_gemm9p_n512.md"},
        {"bytes_per_launch": 1005568 + 0, "src_sha": "881cb10161712188", "n": 220, "N": 113247,
         "capture": "profiles/predict_tc_fp16x3_gemm7p_n220.md"},
    ],
}


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


def tc_mma_flops(n, N):
    """Tensor-core flops the FP16X3 / BF16X3 kernel issues: 3 products, 32-wide
    chunks, each chunk's N range running from its first row to n_pad."""
    n_pad = (n + 31) // 32 * 32
    cols = sum(n_pad - c * 32 for c in range(n_pad // 32))
    return 3 * 2 * 128 * 32 * cols * ((N + 127) // 128)


def traffic_for(key, precision, n, N):
    """Per-launch DRAM bytes from the committed ncu capture of this kernel source
    and launch size, else None."""
    for tr in TRAFFIC.get(key, []):
        if tr["src_sha"] == kernel_sha(precision) and tr["n"] == n and tr["N"] == N:
            return tr["bytes_per_launch"]
    return None


def roofline_for(precision, n, d, N, k1_time):
    alg = float(N) * n * (n + 1)                       # triangular contraction, flops
    if precision == "fp64":
        fl = float(flops_per_candidate(n, d)) * N
        ach = fl / k1_time / 1e12
        return {"bound": "alu", "kernel": "predict_f64_kernel", "achieved": round(ach, 4),
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": round(ach / FP64_PEAK_TFLOPS, 4),
                "peak_source": "nominal GB300 FP64 (recipe table), not measured; ncu: FP64 pipe 93 % busy",
                "traffic": traffic_for("predict_f64", precision, n, N),
                "flops_per_launch": fl, "launch_s": k1_time}
    peaks = _peaks()
    peak = peaks["bf16_tflops"] * (0.5 if precision == "tf32" else 1.0)
    ach = alg / k1_time / 1e12
    issued = (tc_mma_flops(n, N) / (3 if precision == "tf32" else 1)) / k1_time / 1e12
    return {"bound": "tensor", "kernel": "predict_tc_kernel<%s>" % precision, "achieved": round(ach, 2),
            "peak": peak, "unit": "TFLOP/s", "frac": round(ach / peak, 4),
            "peak_source": ("measured bf16 burst (MEASURED_PEAKS.json)" + (" x 1/2 nominal tf32 ratio"
                            if precision == "tf32" else "; f16 runs at the bf16 rate")),
            "mma_issued_tflops": round(issued, 1), "mma_issued_frac": round(issued / peak, 4),
            "traffic": traffic_for("predict_tc_" + precision, precision, n, N),
            "flops_per_launch": alg, "launch_s": k1_time}


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


def batched_workload(count, steps, warm, precision, seed=0):
    """Sessions of the batched configuration: d ~ U{3..9}, N ~ log-U[1k, 500k],
    final n ~ U{20..400}; the last warm + steps observations of each session
    are held back for the timed steps."""
    from paper_2111_14991_gb300 import Batch, Space
    from paper_2111_14991_gb300 import workloads as W
    sps = W.batched_spaces(count, seed=seed)
    spaces, obs = [], []
    n_max = min(512, max(sp.meta["n_obs"] for sp in sps) + 1)
    for sp in sps:
        land = W.Landscape(sp, sp.meta["session"])
        idx = W.clustered_observations(land, sp.meta["n_obs"], sp.meta["session"])
        obs.append((idx, land.clean(idx)))
        spaces.append(Space(sp.grids, sp.invalid, precision=precision, af="ei", n_max=n_max))
    batch = Batch(spaces)
    hold = warm + steps
    rounds = max(len(i) for i, _ in obs) - hold
    for r in range(rounds):                      # initial observations, one batched update per round
        ii = [int(i[r]) if r < len(i) - hold else -1 for i, _ in obs]
        yy = [float(y[r]) if r < len(i) - hold else 0.0 for i, y in obs]
        batch.observe(ii, yy)
    return sps, spaces, batch, obs


def measure_batched(count, steps, warm, precision, stream):
    """Device-timed batched steps: one observation per session (batched update)
    and one prediction pass per session (one persistent launch)."""
    import torch
    sps, spaces, batch, obs = batched_workload(count, steps, warm, precision)
    hold = warm + steps
    times, scored, flops, tune = [], 0, 0.0, None
    for t in range(warm + steps):
        if t == warm:
            tune = batch.autotune(reps=2)        # pipeline shapes of the batched launch
        ii = [int(i[len(i) - hold + t]) for i, _ in obs]
        yy = [float(y[len(y) - hold + t]) for _, y in obs]
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
            n_now = [len(i) - hold + t + 1 for i, _ in obs]
            flops += sum(float(sp.n_valid) * n * (n + 1) for sp, n in zip(sps, n_now))
    launches = batch.launch_count()
    batch.close()
    for sp in spaces:
        sp.close()
    return dict(value=scored / sum(times), times=times, flops=flops, sessions=count,
                candidates=sum(sp.n_valid for sp in sps), launches=launches, tune=tune)


def measure_serving(count, rate, duration, precision, extra=160, seed=0):
    """Open-loop serving: Poisson arrivals at `rate` requests/s (observe one new
    point + suggest) spread uniformly over `count` live sessions of the batched
    configuration's sizes, for `duration` seconds; then a closed-loop run with
    one request of every session always in flight (saturation)."""
    import torch
    from paper_2111_14991_gb300 import Server
    from paper_2111_14991_gb300 import workloads as W
    sps = W.batched_spaces(count, seed=seed)
    srv = Server(budget_bytes=120 << 30, max_sessions=1024)
    rng = np.random.default_rng(seed + 99)
    sids, pending = [], []
    for sp in sps:
        land = W.Landscape(sp, sp.meta["session"])
        init = W.clustered_observations(land, min(sp.meta["n_obs"], 512 - extra - 8), sp.meta["session"])
        rest = np.setdiff1d(rng.choice(sp.n_valid, min(sp.n_valid, len(init) + extra), replace=False), init)
        sid = srv.open(sp.grids, sp.invalid, precision=precision, af="ei", n_max=512)
        for i, v in zip(init, land.clean(init)):
            srv.submit(sid, int(i), float(v), suggest=False)
        sids.append(sid)
        pending.append(list(zip(rest.tolist(), land.clean(rest).tolist())))
    n_warm = srv.stats()["requests"]
    t_end = time.time() + 600
    while srv.stats()["completed"] < n_warm and time.time() < t_end:
        srv.poll(4096, wait_ms=20)
    srv.poll(1 << 16, wait_ms=0)
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
    lat = np.array([c["t_done"] - c["t_submit"] for c in done if c["idx"] >= 0])
    span = max(c["t_done"] for c in done) - t0
    scored = sum(c["info"]["n_scored"] for c in done if c["idx"] >= 0)
    open_loop = {"requests": len(lat), "rate_req_s": rate, "duration_s": round(span, 3),
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
            srv.submit(sids[s], i, v, tag=s)
            inflight += 1
    scored, n_done, t_stop = 0, 0, t0 + duration
    while inflight and srv.now() < t_stop:
        for c in srv.poll(4096, wait_ms=5):
            inflight -= 1
            n_done += 1
            scored += c["info"]["n_scored"]
            s = sids.index(c["session"])
            if pending[s]:
                i, v = pending[s].pop()
                srv.submit(sids[s], i, v, tag=s)
                inflight += 1
    span = srv.now() - t0
    while inflight:
        inflight -= len(srv.poll(4096, wait_ms=20))
    st = srv.stats()
    closed_loop = {"requests": n_done, "duration_s": round(span, 3), "candidates_per_s": round(scored / span, 1),
                   "iterations": st["iterations"] - it0["iterations"]}
    stats = srv.stats()
    srv.close()
    return {"sessions": count, "open_loop": open_loop, "closed_loop": closed_loop,
            "admitted": stats["admitted"], "bytes_in_use": stats["bytes_in_use"]}


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
    for t in range(10 + max(args.latency_reps, steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.suggest()
        if t >= 10:
            lat.append(time.perf_counter() - t0)
    s.close()
    e2e_tot = sum(e2e_t)

    # ---- the other forms on the same GPU (device-timed, same recipe)
    forms = {}
    if not args.no_forms:
        for fcfg, fprec, fsteps in ((2, "fp64", steps), (2, "fp16x3", steps), (3, "fp16x3", steps),
                                    (3, "fp64", 3)):
            if (fcfg, fprec) == (args.config, args.precision):
                continue
            f = measure_device(fcfg, fprec, fsteps, 3, flush, stream)
            forms[f"config{fcfg}/{fprec}"] = {
                "value": round(f["value"], 1), "unit": "candidates/s",
                "ms_per_step": round(1e3 * sum(f["times"]) / len(f["times"]), 4),
                "n_obs": f"{f['n0'] + 4}..{f['n_last']}", "autotune": f["tune"],
                "roofline": roofline_for(fprec, f["n_last"], f["sp"].d, f["sp"].n_valid, f["k1"])}
        if not args.no_serving:
            forms["config5/fp16x3-served"] = measure_serving(args.batch_sessions, 2000.0, 4.0, "fp16x3")
        if not args.no_batched:
            bsteps = max(3, min(steps, 10))
            f = measure_batched(args.batch_sessions, bsteps, 3, "fp16x3", stream)
            peak = _peaks()["bf16_tflops"]
            ach = f["flops"] / sum(f["times"]) / 1e12
            forms["config4/fp16x3-batched"] = {
                "value": round(f["value"], 1), "unit": "candidates/s",
                "ms_per_step": round(1e3 * sum(f["times"]) / len(f["times"]), 4),
                "sessions": f["sessions"], "candidates": f["candidates"], "autotune": f["tune"],
                "what": "per step: one batched update + one batched prediction pass of every session",
                "l2": "working set > L2 (no flush)",
                "roofline": {"bound": "tensor", "kernel": "whole batched step", "achieved": round(ach, 2),
                             "peak": peak, "unit": "TFLOP/s", "frac": round(ach / peak, 4),
                             "peak_source": "measured bf16 burst; step time bounds the kernel time from above",
                             "traffic": None}}

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
        "clocks": clocks,
        "forms": forms,
    }
    return out


def cpu_baseline(cfg_id, budget_s=15.0):
    """The oracle, as it stands, on the host: one suggest's prediction + scores
    over a bounded sample of the candidates at the final state."""
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
    done, t_pred = 0, 0.0
    while t_pred < budget_s:
        sel = rng.choice(sp.n_valid, sample, replace=False)
        t0 = time.perf_counter()
        mu, var = O.gp_posterior(fit, coords[sel])
        sd = np.sqrt(var)
        for af in ("ei", "poi", "lcb"):
            sc = O.acquisition(af, mu, sd, float(np.min((y - y.mean()) / y.std())), 0.1)
            O.masked_topk(sc, np.ones(len(sel), bool), 3)
        t_pred += time.perf_counter() - t0
        done += sample
    cores = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        cores = max(int(i.get("num_threads", 1)) for i in threadpool_info()) or cores
    except Exception:
        pass
    return {"value": round(done / (t_pred + t_fit * done / sp.n_valid), 1), "unit": "candidates/s",
            "cores": cores, "kind": "oracle",
            "sample": f"{done} candidates in batches of {sample} drawn from the {sp.n_valid} at "
                      f"n = {cfg['n_final']} (fit once, {t_pred:.1f} s of prediction + EI/PI/LCB top-3)"}


def run_reference(args):
    import oracle as O
    cfg = CONFIGS[args.config]
    sp = space_for(args.config)
    idx, y = observations(sp, args.config, cfg["n_final"], seed=0)
    coords = sp.valid_coords()
    per_step = max(2000, min(sp.n_valid, 20000))
    rng = np.random.default_rng(2)
    times = []
    for t in range(args.warmup + args.steps):
        n = cfg["n_final"] - (args.steps - t) if t >= args.warmup else cfg["n_final"] - args.steps
        n = max(2, n)
        sel = rng.choice(sp.n_valid, per_step, replace=False)
        t0 = time.perf_counter()
        fit = O.gp_fit(coords[idx[:n]], y[:n], 1.5, 1.5, 1e-10)
        mu, var = O.gp_posterior(fit, coords[sel])
        sd = np.sqrt(var)
        for af in ("ei", "poi", "lcb"):
            O.masked_topk(O.acquisition(af, mu, sd, -1.0, 0.1), np.ones(per_step, bool), 3)
        if t >= args.warmup:
            times.append(time.perf_counter() - t0)
    value = per_step * len(times) / sum(times)
    cores = os.cpu_count()
    out = {"metric": METRIC, "value": round(value, 1), "unit": "candidates/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sum(times) / len(times), 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": cfg["name"], "precision": "fp64 (CPU oracle)"},
           "cpu_baseline": {"value": round(value, 1), "unit": "candidates/s", "cores": cores, "kind": "oracle",
                            "sample": f"{per_step} random candidates per step, fit + predict + 3 AFs"},
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
    ap.add_argument("--latency-reps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the other precision forms")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched (256-session) form")
    ap.add_argument("--batch-sessions", type=int, default=256)
    ap.add_argument("--no-serving", action="store_true", help="skip the served form")
    ap.add_argument("--kernel-only", type=int, default=0,
                    help="only launch the prediction kernel this many times at the final state")
    ap.add_argument("--quality", type=int, default=0,
                    help="run the tuning-quality protocol with this many repeats per BO strategy instead")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
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
        print(json.dumps(out))


if __name__ == "__main__":
    main()
