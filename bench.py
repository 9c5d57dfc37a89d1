"""Benchmark of the k-means|| hot path on GB300 (one JSON line on rank 0).

A step is one pass of the whole path over one synthetic batch: init (Alg. 2
steps 1-2), r rounds of draw + union/update (steps 4-5), weights (step 7),
weighted k-means++ recluster (step 8), then Lloyd's iteration (until no label
changes, at most the workload's cap of updates).  The default workload is the
largest single-GPU configuration: a GAUSSMIXTURE of 10,000 components, n =
10,000,000 points in d = 128 (centers ~ N(0, 100 I)), k = 10,000, l = 2k, r = 5,
Lloyd capped at 10 updates.

value = algorithmic distance evaluations per second over the whole job
(init n, each round n |C'_i|, recluster k m, Lloyd n k per assignment).  The
same line carries the plain FP32 CUDA-core path on the same data and seed
(``fp32_arm``): its time per step, its final cost and the relative difference to
this arm's final cost (the metric compares the two at equal cost).
Multi-GPU runs are independent replicas (one per rank, weak scaling).

--impl reference times the FP64 CPU oracle instead (rank 0 only), on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "k-means|| init+Lloyd s and dist-evals/s, BF16/FP8+refine vs FP32 at equal cost"
UNIT = "dist-evals/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
SMS = 152
FP32_LANES_PER_SM = 128


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["source"] = "fallback"
    return d


def workload(args):
    from paper_1203_6402_gb300 import datagen
    w = dict(datagen.WORKLOADS[args.workload])
    if args.n:
        w["n"] = args.n
    if args.ell_factor:
        w["ell"] = args.ell_factor * w["k"]
    return w


def default_precision(name: str) -> str:
    """Split BF16 where its K = 3d + 2 fits the screening kernel (d <= 62), else plain BF16."""
    from paper_1203_6402_gb300 import datagen
    d = datagen.WORKLOADS[name]["d"]
    return "bf16x3" if 3 * d + 2 <= 192 else "bf16"


def count_dist_evals(n, k, stats, lloyd_iters):
    """Algorithmic distance evaluations of one step (no padding, no refinement)."""
    init = n
    rounds = n * sum(stats["round_added"])
    recluster = k * stats["m"]
    lloyd = (lloyd_iters + 1) * n * k
    return init + rounds + recluster + lloyd, dict(init=init, rounds=rounds, recluster=recluster, lloyd=lloyd)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index: int):
        self.proc = None
        self.dev = dev_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return self.parse(out)

    @staticmethod
    def parse(out: str):
        """Median SM clock, maximum clock and the throttle reasons seen in the CSV
        lines of ``nvidia-smi --query-gpu=FIELDS --format=csv,noheader,nounits``."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ our arm
def _phase_events(torch, stream, names):
    ev = {nm: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for nm in names}
    return ev


def run_step(km, torch, X, k, ell, rounds, seed, prec, stream, sampling, max_iter, timing=False, phases=None,
             recluster_batch=0):
    """One pass of the whole path through the C ABI; returns (stats, lloyd output)."""
    def mark(nm, i):
        if phases is not None:
            phases[nm][i].record(stream)
    mark("init", 0)
    g = km.KMeansPar(X, k, ell, rounds, seed=seed, precision=prec, stream=stream, sampling=sampling,
                     recluster_batch=recluster_batch)
    if timing:
        km.kmpar_set_timing(g.ctx, True)
    mark("init", 1)
    mark("rounds", 0)
    for i in range(1, rounds + 1):
        g.round(i)
    mark("rounds", 1)
    mark("weight", 0)
    g.weight()
    mark("weight", 1)
    mark("recluster", 0)
    C, _ = g.recluster()
    mark("recluster", 1)
    mark("lloyd", 0)
    out = g.lloyd(C, max_iter, labels=True)
    mark("lloyd", 1)
    st = g.stats()
    g.close()
    return st, out


def traffic_record(kernel: str, workload: str, precision: str):
    """DRAM bytes per launch of `kernel` from a committed ncu summary, used only
    while the kernel's source is the one that was captured (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.md")
    src = os.path.join(ROOT, "paper_1203_6402_gb300", "csrc", "nearest_tc_kernel.cuh")
    if not (os.path.exists(path) and os.path.exists(src)):
        return None, None
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()[:16]
    with open(path) as f:
        for line in f:
            parts = [p.strip() for p in line.strip().strip("|").split("|")]
            if len(parts) >= 5 and parts[0] == kernel and parts[1] == workload and parts[2] == precision:
                try:
                    val = float(parts[3])
                except ValueError:
                    continue
                return (val, parts[4]) if parts[4] == sha else (None, parts[4])
    return None, None


def run_batched(args, rank, world):
    """The batched configuration: 4,096 independent GAUSSMIXTURE problems (n and k
    log-uniform in [1e3, 2e5] and [16, 256], d in {32, 64, 128}, l = 2k, r = 5,
    10 Lloyd updates) in one kmpar_batch_run call per step.  The points of each
    problem are drawn on the device from the problem's own seed (same recipe as
    datagen.gauss_mixture; the full batch is ~46 GB)."""
    import torch
    from paper_1203_6402_gb300 import datagen
    from paper_1203_6402_gb300 import kmpar as km

    km.load()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    count = args.batch_count
    probs = datagen.batched_problems(count, seed=1000 + rank)
    total = sum(p["n"] * p["d"] for p in probs)
    X = torch.empty(total, dtype=torch.float32, device=dev)
    gen = torch.Generator(device=dev)
    for p in probs:
        gen.manual_seed(p["data_seed"])
        n, d, k = p["n"], p["d"], p["k"]
        cen = torch.randn(k, d, generator=gen, device=dev) * (10.0 ** 0.5)
        comp = torch.randint(0, k, (n,), generator=gen, device=dev)
        X[p["x_offset"]: p["x_offset"] + n * d].view(n, d).copy_(cen[comp] + torch.randn(n, d, generator=gen,
                                                                                           device=dev))
    C = torch.empty(sum(p["k"] * p["d"] for p in probs), dtype=torch.float32, device=dev)
    L = torch.empty(sum(p["n"] for p in probs), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    # the schedule the autotuner measured fastest (paper_1203_6402_gb300/batch_tune.py)
    from paper_1203_6402_gb300 import batch_tune
    table = batch_tune.load_table()
    if table is not None:
        km.kmpar_batch_set_split(int(table["rows_per_block"]))

    def step():
        st, res = km.kmpar_batch_run(X.data_ptr(), probs, C.data_ptr(), L.data_ptr(), stream=stream.cuda_stream)
        assert st in (km.KMPAR_OK, km.KMPAR_WARN_FEW_CANDIDATES), st
        return res

    def evals_of(res):
        tot = 0
        for p, r in zip(probs, res):
            n, k = p["n"], p["k"]
            tot += n + n * (r["m"] - 1) + k * r["m"] + (r["iters"] + 1) * n * k
        return tot

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()
    evals = evals_of(res)
    barrier(world)
    sampler = ClockSampler(local)
    sampler.start()
    l0 = km.kmpar_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    tot = 0
    for _ in range(args.steps):
        tot += evals_of(step())
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = km.kmpar_launch_count() - l0
    clocks = sampler.stop()
    ms = allreduce_max(ev0.elapsed_time(ev1), world)
    value = allreduce_sum(float(tot), world) / (ms / 1e3)
    # end to end: points from pinned host memory, centers and labels back, every step
    e2e = None
    try:
        Xh = X.cpu().pin_memory()
        Ch = torch.empty(C.numel(), dtype=torch.float32).pin_memory()
        Lh = torch.empty(L.numel(), dtype=torch.int32).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_steps = max(1, min(args.steps, 3))
        for _ in range(e2e_steps):
            X.copy_(Xh, non_blocking=True)
            step()
            Ch.copy_(C, non_blocking=True)
            Lh.copy_(L, non_blocking=True)
        torch.cuda.synchronize()
        e2e_s = allreduce_max(time.perf_counter() - t0, world)
        e2e = {"value": allreduce_sum(float(evals * e2e_steps), world) / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": total * 4, "d2h_bytes_per_step": C.numel() * 4 + L.numel() * 4,
               "steps": e2e_steps, "path": "torch copies around kmpar_batch_run (device pointers)"}
        del Xh, Ch, Lh
    except RuntimeError as exc:   # pinned host memory for the whole batch may not be available
        e2e = {"value": None, "unit": UNIT, "note": f"no end-to-end figure: {exc}"[:200]}
    # FP32 CUDA-core issue roofline: 2 instructions (sub, fma) per padded coordinate
    peaks = load_peaks()
    clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    instr = 0.0
    for p, r in zip(probs, res):
        dp = 32 if p["d"] <= 32 else (64 if p["d"] <= 64 else 128)
        n, k = p["n"], p["k"]
        instr += 2.0 * dp * (n + n * (r["m"] - 1) + k * r["m"] + (r["iters"] + 1) * n * k)
    achieved = instr / (ms / args.steps / 1e3) / 1e12
    peak = FP32_LANES_PER_SM * SMS * clk / 1e12
    xbytes = total * 4
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (exact difference form on CUDA cores), f64 sums", "data": "synthetic",
        "config": {"workload": (f"batched: {count} GAUSSMIXTURE problems, n log-uniform [1e3, 2e5], "
                                f"d in {{32, 64, 128}}, k log-uniform [16, 256], l = 2k, r = 5, 10 Lloyd updates; "
                                f"one kmpar_batch_run per step (one block per problem, largest first)"),
                   "sum_n": int(sum(p["n"] for p in probs)), "x_gb": xbytes / 1e9,
                   "schedule": ({"rows_per_block": table["rows_per_block"], "source": "batch_tuning.json"}
                                if table is not None else {"rows_per_block": 25000, "source": "default"}),
                   "parallelism": f"replicas x{world}", "l2": f"inputs larger than L2 (X {xbytes / 1e9:.1f} GB)"},
        "dist_evals_per_step": evals, "gpu_launches": int(launches), "e2e": e2e,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinstr/s (FP32 issue)",
                     "frac": achieved / peak, "traffic": None, "kernel": "batch_kernel (all problems)",
                     "peak_source": f"derived: 128 FP32 lanes x 152 SMs x {peaks.get('sm_max_mhz', 2070.0)} MHz",
                     "hbm": {"gbs_min": xbytes * 16 / (ms / args.steps / 1e3) / 1e9,
                             "note": "X read once per pass, 16 passes (init, 5 rounds, 10+1 Lloyd)",
                             "peak_gbs": peaks.get("hbm_gbs")}},
        "clocks": clocks,
        "problems": {"status_counts": {str(s): sum(1 for r in res if r["status"] == s) for s in
                                       sorted(set(r["status"] for r in res))},
                     "lloyd_iters_mean": statistics.mean(r["iters"] for r in res)},
        **({"cpu_baseline": cpu_baseline_batched(args)} if rank == 0 and world == 1 and not args.no_cpu_baseline
           else {}),
    }


def run_ours(args, rank, world):
    import torch
    from paper_1203_6402_gb300 import datagen
    from paper_1203_6402_gb300 import kmpar as km

    km.load()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args)
    n, k, ell, rounds, max_iter = w["n"], w["k"], w["ell"], w["rounds"], w["max_iter"]
    data_seed = 1000 + rank
    Xh = datagen.make(args.workload, seed=data_seed, n=n)
    d = Xh.shape[1]
    X = torch.from_numpy(Xh).to(dev)
    stream = torch.cuda.current_stream()
    prec = km.PRECISIONS[args.precision]
    seed = 7 + rank

    def step(timing=False, phases=None, precision=prec):
        return run_step(km, torch, X, k, ell, rounds, seed, precision, stream, args.sampling, max_iter, timing, phases,
                        args.recluster_batch)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # one timed step with the kernel-level and phase events, outside the job timer
    phases = _phase_events(torch, stream, ["init", "rounds", "weight", "recluster", "lloyd"])
    st_t, out_t = step(timing=True, phases=phases)
    torch.cuda.synchronize()
    phase_ms = {nm: a.elapsed_time(b) for nm, (a, b) in phases.items()}
    evals, parts = count_dist_evals(n, k, st_t, out_t["iters"])

    barrier(world)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = km.kmpar_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    total_evals = 0
    kern = {"round": [0.0, 0], "assign": [0.0, 0]}
    iters, finals = [], []
    for _ in range(args.steps):
        st, out = step(timing=True)
        e, _ = count_dist_evals(n, k, st, out["iters"])
        total_evals += e
        kern["round"][0] += st["kernel_ms"][0]; kern["round"][1] += st["kernel_launches"][0]
        kern["assign"][0] += st["kernel_ms"][1]; kern["assign"][1] += st["kernel_launches"][1]
        iters.append(out["iters"])
        finals.append(out["final_cost"])
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = km.kmpar_launch_count() - l0
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max = allreduce_max(ms, world)
    evals_all = allreduce_sum(float(total_evals), world)
    value = evals_all / (ms_max / 1e3)

    # end to end through the public API with host buffers (pinned), copies inside the timer
    Xpin = torch.from_numpy(Xh).pin_memory()
    fit_flags = (km.KMPAR_EXACT_SAMPLING if args.sampling == "exact" else 0) | (args.recluster_batch << 16)
    Cpin = torch.empty(k, d, dtype=torch.float32).pin_memory()
    Lpin = torch.empty(n, dtype=torch.int32).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_evals = 0
    for _ in range(e2e_steps):
        r = km.kmpar_fit(Xpin.data_ptr(), n, d, k, ell, rounds, seed, prec, max_iter, Cpin.data_ptr(),
                         Lpin.data_ptr(), flags=km.KMPAR_HOST_BUFFERS | fit_flags, stream=stream.cuda_stream)
        assert r["iters"] == out_t["iters"], "end-to-end run took a different trajectory"
        e2e_evals += evals
    torch.cuda.synchronize()
    e2e_s = allreduce_max(time.perf_counter() - t0, world)
    e2e_value = allreduce_sum(float(e2e_evals), world) / e2e_s
    del Xpin, Cpin, Lpin

    # the plain FP32 CUDA-core path on the same data and seed: the metric's comparison arm
    fp32_arm = None
    if args.precision != "fp32" and args.fp32_steps > 0:
        for _ in range(args.fp32_warmup):
            step(precision=km.KMPAR_FP32)
        torch.cuda.synchronize()
        fa, fb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fa.record(stream)
        f_out, f_st = [], None
        for _ in range(args.fp32_steps):
            f_st, o = step(precision=km.KMPAR_FP32)
            f_out.append(o)
        fb.record(stream)
        torch.cuda.synchronize()
        f_ms = fa.elapsed_time(fb) / args.fp32_steps
        f_evals, _ = count_dist_evals(n, k, f_st, f_out[-1]["iters"])
        f_cost = f_out[-1]["final_cost"]
        fp32_arm = {"ms_per_step": f_ms, "value": f_evals / (f_ms / 1e3), "unit": UNIT,
                    "steps": args.fp32_steps, "warmup": args.fp32_warmup,
                    "final_cost": f_cost, "candidates": f_st["m"], "lloyd_iters": f_out[-1]["iters"],
                    "final_cost_rel_diff": abs(out_t["final_cost"] - f_cost) / max(abs(f_cost), 1e-300),
                    "equal_cost": abs(out_t["final_cost"] - f_cost) <= 1e-4 * abs(f_cost),
                    "same_decisions": (out_t["final_cost"] == f_cost and st_t["m"] == f_st["m"]
                                       and out_t["iters"] == f_out[-1]["iters"]),
                    "speedup": f_ms / (ms_max / args.steps)}

    # roofline of the dominant kernel (the distance pass with the most time)
    peaks = load_peaks()
    cls = max(kern, key=lambda c: kern[c][0])
    kms, kl = kern[cls]
    per_launch_ms = kms / max(kl, 1)
    if cls == "assign":
        units = n * k                              # dist-evals per Lloyd assignment pass
        centers_per_pass = k
    else:
        centers_per_pass = sum(st_t["round_added"]) / max(len(st_t["round_added"]), 1)
        units = n * centers_per_pass
    clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    secs = per_launch_ms / 1e3
    if args.precision == "fp32":
        # exact FP32 difference form on CUDA cores: 2 FP32 instructions (sub, fma) per
        # coordinate; peak = 128 FP32 lanes x 152 SMs x max SM clock
        achieved = units * 2 * d / secs / 1e12
        peak = FP32_LANES_PER_SM * SMS * clk / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinstr/s (FP32 issue)",
                    "frac": achieved / peak, "traffic": None, "kernel": f"nearest_kernel ({cls} pass)",
                    "peak_source": f"derived: 128 FP32 lanes x 152 SMs x {peaks.get('sm_max_mhz', 2070.0)} MHz"}
    else:
        # tcgen05 screening: achieved = algorithmic GEMM-form flops 2 d per distance; the
        # kernel is timed inside a long step, so the peak is the measured sustained figure
        # for its operand type (FP8 = 2 x BF16, the nominal ratio)
        tflops = units * 2 * d / secs / 1e12
        ratio = 2.0 if args.precision == "fp8" else 1.0
        peak = ratio * float(peaks.get("bf16_tflops_sustained", PEAKS_FALLBACK["bf16_tflops_sustained"]))
        kk, bn = screen_shape(args.precision, d)
        npad, kpad = -(-n // 128) * 128, -(-int(centers_per_pass) // bn) * bn
        exec_tflops = 2.0 * npad * kpad * kk / secs / 1e12
        kernel_name = "tc::nearest_tc_kernel"
        traffic, cap_sha = traffic_record(f"{kernel_name} ({cls})", args.workload, args.precision) \
            if not args.n else (None, None)
        roofline = {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                    "frac": tflops / peak, "traffic": traffic,
                    "kernel": f"{kernel_name} ({cls} pass)",
                    "peak_source": (f"{peaks.get('source')} bf16 sustained" + (" x 2 (FP8 nominal ratio)"
                                    if ratio == 2.0 else "") + " (kernel timed inside the step)"),
                    "executed": {"tflops": exec_tflops, "frac": exec_tflops / peak,
                                 "note": "MMA flops issued: K and the center count padded to the tile"},
                    "hbm": {"gbs": (traffic or 0) / secs / 1e9, "peak_gbs": peaks.get("hbm_gbs")}}
        if traffic is None:
            roofline["traffic_note"] = ("no ncu capture of the current kernel source" if cap_sha is None else
                                        f"capture taken on kernel source {cap_sha}, which has changed since")
    roofline.update({"avg_launch_ms": per_launch_ms, "launches": kl,
                     "classes": {c: {"ms": kern[c][0], "launches": kern[c][1],
                                     "avg_launch_ms": kern[c][0] / max(kern[c][1], 1)} for c in kern}})

    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.precision],
        "data": "synthetic",
        "config": {"workload": (f"{args.workload}: n={n} d={d} k={k} l={ell:g} r={rounds}, "
                                f"Lloyd until no label changes, capped at {max_iter} updates"),
                   "precision": args.precision, "sampling": args.sampling,
                   "recluster_batch": args.recluster_batch,
                   "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2 (X {n * d * 4 / 1e6:.0f} MB > 129 MB)"},
        "init_lloyd_s": ms_max / args.steps / 1e3,
        "dist_evals_per_step": evals, "dist_evals_parts": parts,
        "phase_ms": phase_ms, "recluster_ms": phase_ms["recluster"],
        "lloyd_iters": iters, "final_cost": out_t["final_cost"], "candidates": st_t["m"],
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * d * 4,
                "d2h_bytes_per_step": k * d * 4 + n * 4, "steps": e2e_steps},
        "fp32_arm": fp32_arm,
        "roofline": roofline, "clocks": clocks,
        "refine": {key: st_t[key] for key in ("sample_near", "sample_refined", "argmin_fp64", "argmin_wide",
                                             "screen_rows", "screen_fallback", "screen_exact",
                                             "recluster_near", "recluster_snapshots", "lloyd_settled")},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(args)
    return res


def screen_shape(precision: str, d: int):
    """(K elements the MMA executes, centers per tile) of the screening pass, as the
    library chooses them: K bytes per row for the format (BF16 adds two norm columns
    unless they would cost a 128-byte K atom, then the norms go to the epilogue),
    MMAs of 32 bytes of K, 256-wide center tiles up to two K atoms and 128-wide beyond."""
    if precision == "bf16x3":
        kbytes, esz = 2 * (3 * d + 2), 2
    elif precision == "fp8":
        kbytes, esz = d, 1
    else:
        kbytes = 2 * (d + 2)
        if (d + 2 + 63) // 64 > (d + 63) // 64:
            kbytes = 2 * d
        esz = 2
    katoms = (kbytes + 127) // 128
    kk = (kbytes + 31) // 32 * (32 // esz)
    bn = 256 if katoms <= 2 else 128
    return kk, bn


DTYPES = {"fp32": "f32",
          "bf16": "bf16 screening, f32 refine, f64 sums",
          "bf16x3": "bf16 (split hi/lo) screening, f32 refine, f64 sums",
          "fp8": "fp8 e4m3 (per-row scaled) screening, f32 refine, f64 sums"}


# ------------------------------------------------------------------ CPU oracle arms
def oracle_sample(args):
    """A bounded sample of the workload for the FP64 oracle: the same generator and
    dimension, n_s points and k_s = k n_s / n clusters (the workload's points per
    cluster; at least 10), l_s = l k_s / k, the same r, Lloyd capped at the
    --cpu-lloyd-iters updates."""
    w = workload(args)
    n_s = min(args.cpu_sample_n, w["n"])
    k_s = max(10, min(w["k"], int(round(w["k"] * n_s / w["n"]))))
    ell_s = w["ell"] * k_s / w["k"]
    return dict(n=n_s, k=k_s, ell=ell_s, rounds=w["rounds"], lloyd=args.cpu_lloyd_iters)


def _oracle_job(argv):
    """Runs in a child process: one oracle pass of the sample; (seconds, dist-evals, info)."""
    root, wname, smp, data_seed, run_seed, sampling, rbatch = argv
    if root not in sys.path:
        sys.path.insert(0, root)
    from oracle import oracle
    from paper_1203_6402_gb300 import datagen
    w = datagen.WORKLOADS[wname]
    if w["kind"] == "gmm":
        Xs = datagen.gauss_mixture(smp["n"], w["d"], smp["k"], w["R"], data_seed)
    else:
        Xs = datagen.kdd_like(smp["n"], data_seed)
    t0 = time.perf_counter()
    par = oracle.kmeans_par(Xs, smp["k"], smp["ell"], smp["rounds"], seed=run_seed, sampling=sampling,
                            recluster_batch=rbatch)
    _, _, it, _, _, _ = oracle.lloyd(Xs, par.seed_centers, smp["lloyd"])
    dt = time.perf_counter() - t0
    n_s, k_s = smp["n"], smp["k"]
    evals = n_s + n_s * (len(par.cand) - 1) + k_s * len(par.cand) + (it + 1) * n_s * k_s
    return dt, evals, dict(lloyd_iters=it, candidates=len(par.cand))


def _sample_text(args, smp, threads):
    w = workload(args)
    return (f"FP64 C oracle, {threads}: same generator (d={w['d']}), n={smp['n']} points, "
            f"k={smp['k']} (the workload's {w['n'] // w['k']} points per cluster), l={smp['ell']:g}, "
            f"r={smp['rounds']}, Lloyd capped at {smp['lloyd']} updates")


def _oracle_batched_job(argv):
    """Child process: the oracle on a seeded subset of batched problems; (seconds, dist-evals)."""
    root, seed, count, n_hi = argv
    if root not in sys.path:
        sys.path.insert(0, root)
    from oracle import oracle
    from paper_1203_6402_gb300 import datagen
    probs = datagen.batched_problems(count, seed=seed, n_hi=n_hi)
    X = datagen.batched_points(probs)
    t0 = time.perf_counter()
    ev = 0
    for p in probs:
        n, d, k = p["n"], p["d"], p["k"]
        Xi = X[p["x_offset"]: p["x_offset"] + n * d].reshape(n, d)
        par = oracle.kmeans_par(Xi, k, p["ell"], p["rounds"], seed=p["seed"])
        _, _, it, _, _, _ = oracle.lloyd(Xi, par.seed_centers, p["max_iter"])
        ev += n + n * (len(par.cand) - 1) + k * len(par.cand) + (it + 1) * n * k
    return time.perf_counter() - t0, ev


def cpu_baseline_batched(args, count=12, n_hi=20000):
    import multiprocessing as mp
    from oracle import oracle
    oracle.build()
    dt, ev = _oracle_batched_job((ROOT, 1000, count, n_hi))
    text = (f"FP64 C oracle, {{}}: {count} problems of the batched recipe with n capped at {n_hi} "
            f"(n log-uniform [1e3, {n_hi}], d in {{{{32, 64, 128}}}}, k log-uniform [16, 256], l = 2k, r = 5, "
            f"10 Lloyd updates)")
    res = {"value": ev / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "seconds": dt,
           "sample": text.format("1 thread")}
    cores = os.cpu_count() or 1
    if cores > 1 and not args.no_cpu_all_cores:
        ctx = mp.get_context("spawn")
        t0 = time.perf_counter()
        with ctx.Pool(cores) as pool:
            outs = pool.map(_oracle_batched_job, [(ROOT, 2000 + j, count, n_hi) for j in range(cores)])
        wall = time.perf_counter() - t0
        res["all_cores"] = {"value": sum(o[1] for o in outs) / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "seconds": wall, "sample": text.format(f"{cores} processes x 1 thread") +
                            ", one seeded subset per process; wall time includes process start-up"}
    return res


def cpu_baseline(args):
    """The oracle as it stands: one process (1 thread), then one process per host
    core each on its own seeded sample (all cores busy; it is single-threaded)."""
    import multiprocessing as mp
    from oracle import oracle
    oracle.build()
    smp = oracle_sample(args)
    dt, evals, info = _oracle_job((ROOT, args.workload, smp, 1000, 7, args.sampling, args.recluster_batch))
    res = {"value": evals / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "seconds": dt,
           "sample": _sample_text(args, smp, "1 thread") + f" ({info['lloyd_iters']} updates made, "
                                                          f"{info['candidates']} candidates)"}
    cores = os.cpu_count() or 1
    if cores > 1 and not args.no_cpu_all_cores:
        ctx = mp.get_context("spawn")
        jobs = [(ROOT, args.workload, smp, 1000 + j, 7 + j, args.sampling, args.recluster_batch)
                for j in range(cores)]
        t0 = time.perf_counter()
        with ctx.Pool(cores) as pool:
            outs = pool.map(_oracle_job, jobs)
        wall = time.perf_counter() - t0
        tot = sum(o[1] for o in outs)
        res["all_cores"] = {"value": tot / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "seconds": wall,
                            "sample": _sample_text(args, smp, f"{cores} processes x 1 thread") +
                            ", one seeded sample per process; wall time includes process start-up"}
    return res


def run_reference(args, rank, world):
    from oracle import oracle
    oracle.build()
    if args.workload == "batched":
        for _ in range(args.warmup):
            _oracle_batched_job((ROOT, 1000, 4, 20000))
        tot_t, tot_e = 0.0, 0
        for _ in range(args.steps):
            dt, e = _oracle_batched_job((ROOT, 1000, 4, 20000))
            tot_t += dt
            tot_e += e
        value = tot_e / tot_t
        sample = ("FP64 C oracle, 1 thread, per step: 4 problems of the batched recipe with n capped at 20000")
        return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": "batched (bounded sample)", "precision": "fp64"},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    smp = oracle_sample(argparse.Namespace(**{**vars(args), "cpu_sample_n": args.ref_sample_n}))
    for _ in range(args.warmup):
        _oracle_job((ROOT, args.workload, smp, 1000, 7, args.sampling, args.recluster_batch))
    tot_t, tot_e = 0.0, 0
    for _ in range(args.steps):
        dt, e, _ = _oracle_job((ROOT, args.workload, smp, 1000, 7, args.sampling, args.recluster_batch))
        tot_t += dt
        tot_e += e
    value = tot_e / tot_t
    sample = _sample_text(args, smp, "1 thread") + ", per step"
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload} (bounded sample)", "precision": "fp64",
                   "sampling": args.sampling, "recluster_batch": args.recluster_batch},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ------------------------------------------------------------------ distributed helpers
def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce_device():
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def allreduce_max(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", default=None, choices=["fp32", "bf16", "bf16x3", "fp8"],
                    help="screening arithmetic (default: the fastest one built for the workload's d)")
    ap.add_argument("--workload", default="gmm_n10M_d128_k10000")
    ap.add_argument("--recluster-batch", type=int, default=64,
                    help="step 8: draws per D^2 snapshot (batched rejection form); 0: one draw at a time")
    ap.add_argument("--sampling", default="bernoulli", choices=["bernoulli", "exact"],
                    help="round draws: independent (Alg. 2 step 4) or exactly l per round (Sec. 5.3)")
    ap.add_argument("--n", type=int, default=0, help="override n (same recipe)")
    ap.add_argument("--ell-factor", type=float, default=0.0, help="override l as a multiple of k")
    ap.add_argument("--cpu-sample-n", type=int, default=50000)
    ap.add_argument("--ref-sample-n", type=int, default=20000)
    ap.add_argument("--cpu-lloyd-iters", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-all-cores", action="store_true")
    ap.add_argument("--fp32-steps", type=int, default=1, help="timed steps of the FP32 comparison arm (0: off)")
    ap.add_argument("--fp32-warmup", type=int, default=1)
    ap.add_argument("--batch-count", type=int, default=4096, help="problems of the batched workload")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "fp32" if args.workload == "batched" else default_precision(args.workload)
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    res = run_batched(args, rank, world) if args.workload == "batched" else run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
