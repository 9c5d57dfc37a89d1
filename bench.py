"""Benchmark of the k-means|| hot path on GB300 (one JSON line on rank 0).

A step is one pass of the whole path over one synthetic batch: init (Alg. 2
steps 1-2), r rounds of draw + union/update (steps 4-5), weights (step 7),
weighted k-means++ recluster (step 8), then Lloyd's iteration to a stable
assignment (at most max_iter updates).  The default workload is the
KDDCUP1999-shaped stand-in n = 1,000,000, d = 42, k = 500, l = 2k, r = 5.

value = algorithmic distance evaluations per second over the whole job
(init n, each round n |C'_i|, recluster k m, Lloyd n k per assignment).
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
ALU_LANES_PER_SM = 64          # integer/min-max/logic pipe: half the FP32 lane count
# screening epilogue: per 8 distances 4 pair minima + 4 key builds + 10 top-2 min/max
# = 2.25 ALU ops per distance
SCREEN_ALU_OPS = 2.25
# DRAM bytes (read + write) per launch of the tensor assignment pass, from an ncu capture of the
# same kernel on this workload; to be set to None whenever the kernel changes until it is
# captured again
TC_ASSIGN_TRAFFIC = {"bf16x3": 256.201e6 + 8.731e6}


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

    def step(timing=False):
        g = km.KMeansPar(X, k, ell, rounds, seed=7 + rank, precision=prec, stream=stream, sampling=args.sampling)
        if timing:
            km.kmpar_set_timing(g.ctx, True)
        for i in range(1, rounds + 1):
            g.round(i)
        g.weight()
        C, _ = g.recluster()
        out = g.lloyd(C, max_iter, labels=True)
        st = g.stats()
        g.close()
        return st, out

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # one timed step with the kernel-level events, outside the job timer
    st_t, out_t = step(timing=True)
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
    iters = []
    for _ in range(args.steps):
        st, out = step(timing=True)
        e, _ = count_dist_evals(n, k, st, out["iters"])
        total_evals += e
        kern["round"][0] += st["kernel_ms"][0]; kern["round"][1] += st["kernel_launches"][0]
        kern["assign"][0] += st["kernel_ms"][1]; kern["assign"][1] += st["kernel_launches"][1]
        iters.append(out["iters"])
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
    fit_flags = km.KMPAR_EXACT_SAMPLING if args.sampling == "exact" else 0
    Cpin = torch.empty(k, d, dtype=torch.float32).pin_memory()
    Lpin = torch.empty(n, dtype=torch.int32).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_evals = 0
    for _ in range(e2e_steps):
        r = km.kmpar_fit(Xpin.data_ptr(), n, d, k, ell, rounds, 7 + rank, prec, max_iter, Cpin.data_ptr(),
                         Lpin.data_ptr(), flags=km.KMPAR_HOST_BUFFERS | fit_flags, stream=stream.cuda_stream)
        assert r["iters"] == out_t["iters"], "end-to-end run took a different trajectory"
        e2e_evals += evals
    torch.cuda.synchronize()
    e2e_s = allreduce_max(time.perf_counter() - t0, world)
    e2e_value = allreduce_sum(float(e2e_evals), world) / e2e_s

    # roofline of the dominant kernel (the distance pass with the most time)
    peaks = load_peaks()
    cls = max(kern, key=lambda c: kern[c][0])
    kms, kl = kern[cls]
    per_launch_ms = kms / max(kl, 1)
    if cls == "assign":
        units = n * k                              # dist-evals per Lloyd assignment pass
    else:
        units = n * (sum(st_t["round_added"]) / max(len(st_t["round_added"]), 1))
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
        # tcgen05 screening: the MMA path binds (ncu: tensor pipe ~45% active, ALU ~62%; an
        # instrumented copy shows the epilogue waiting on the accumulator every tile).
        # achieved = algorithmic GEMM-form flops 2 d per distance; the kernel is timed inside a
        # long step, so the peak is the measured sustained BF16 figure
        tflops = units * 2 * d / secs / 1e12
        peak = float(peaks.get("bf16_tflops_sustained", PEAKS_FALLBACK["bf16_tflops_sustained"]))
        # what the tensor cores execute: 3 split products (K = 3 d + 2 padded to 16) for every
        # padded 128-row x 256-column tile
        kk = ((3 * d + 2 if args.precision == "bf16x3" else d + 2) + 15) // 16 * 16
        bn = 256 if kk <= 128 else 128
        npad, kpad = -(-n // 128) * 128, -(-int(units // n) // bn) * bn
        exec_tflops = 2.0 * npad * kpad * kk / secs / 1e12
        alu = units * SCREEN_ALU_OPS / secs / 1e12
        alu_peak = ALU_LANES_PER_SM * SMS * clk / 1e12
        traffic = TC_ASSIGN_TRAFFIC.get(args.precision) if cls == "assign" and args.workload == "kdd_n1M_d42_k500" \
            and not args.n else None
        roofline = {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                    "frac": tflops / peak, "traffic": traffic,
                    "kernel": f"nearest_tc_kernel ({cls} pass)",
                    "peak_source": f"{peaks.get('source')} bf16 sustained (kernel timed inside the step)",
                    "executed": {"tflops": exec_tflops, "frac": exec_tflops / peak,
                                 "note": "MMA flops issued: split products, K and k padded"},
                    "alu": {"achieved": alu, "peak": alu_peak, "unit": "T ALU ops/s", "frac": alu / alu_peak,
                            "peak_source": f"derived: 64 ALU lanes x 152 SMs x {peaks.get('sm_max_mhz', 2070.0)} MHz"},
                    "hbm": {"gbs": (traffic or 0) / secs / 1e9, "peak_gbs": peaks.get("hbm_gbs")}}
    roofline.update({"avg_launch_ms": per_launch_ms, "launches": kl})

    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "bf16 (split hi/lo) screening, f32 refine, f64 sums",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: n={n} d={d} k={k} l={ell:g} r={rounds} Lloyd<={max_iter}",
                   "precision": args.precision, "sampling": args.sampling,
                   "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2 (X {n * d * 4 / 1e6:.0f} MB > 129 MB)"},
        "init_lloyd_s": ms_max / args.steps / 1e3,
        "dist_evals_per_step": evals, "dist_evals_parts": parts,
        "lloyd_iters": iters, "final_cost": out_t["final_cost"], "candidates": st_t["m"],
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * d * 4,
                "d2h_bytes_per_step": k * d * 4 + n * 4, "steps": e2e_steps},
        "roofline": roofline, "clocks": clocks,
        "refine": {key: st_t[key] for key in ("sample_near", "sample_refined", "argmin_fp64", "argmin_wide",
                                             "screen_rows", "screen_fallback",
                                             "recluster_near")},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(args, seconds_hint=20)
    return res


# ------------------------------------------------------------------ CPU oracle arms
def oracle_sample_run(args, n_s: int, lloyd_iters: int):
    """The oracle on a bounded sample of the workload; returns (seconds, dist-evals)."""
    from oracle import oracle
    from paper_1203_6402_gb300 import datagen
    w = workload(args)
    k, ell, rounds = w["k"], w["ell"], w["rounds"]
    Xs = datagen.make(args.workload, seed=1000, n=n_s)
    t0 = time.perf_counter()
    par = oracle.kmeans_par(Xs, k, ell, rounds, seed=7, sampling=getattr(args, "sampling", "bernoulli"))
    _, _, it, _, _, _ = oracle.lloyd(Xs, par.seed_centers, lloyd_iters)
    dt = time.perf_counter() - t0
    evals = n_s + n_s * (len(par.cand) - 1) + k * len(par.cand) + (it + 1) * n_s * k
    return dt, evals, dict(n=n_s, k=k, l=ell, r=rounds, lloyd_iters=it, candidates=len(par.cand))


def cpu_baseline(args, seconds_hint: float = 20.0):
    from oracle import oracle
    oracle.build()
    n_s = args.cpu_sample_n
    dt, evals, info = oracle_sample_run(args, n_s, args.cpu_lloyd_iters)
    return {"value": evals / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "seconds": dt,
            "sample": (f"FP64 C oracle, 1 thread: same generator, n={info['n']} of the workload's points, "
                       f"k={info['k']}, l={info['l']:g}, r={info['r']}, Lloyd capped at "
                       f"{args.cpu_lloyd_iters} updates ({info['lloyd_iters']} made), {info['candidates']} candidates")}


def run_reference(args, rank, world):
    from oracle import oracle
    oracle.build()
    n_s = args.ref_sample_n
    for _ in range(args.warmup):
        oracle_sample_run(args, n_s, args.cpu_lloyd_iters)
    tot_t, tot_e = 0.0, 0
    info = None
    for _ in range(args.steps):
        dt, e, info = oracle_sample_run(args, n_s, args.cpu_lloyd_iters)
        tot_t += dt
        tot_e += e
    value = tot_e / tot_t
    w = workload(args)
    sample = (f"FP64 C oracle, 1 thread, per step: n={n_s} points of the workload's generator, k={w['k']}, "
              f"l={w['ell']:g}, r={w['rounds']}, Lloyd capped at {args.cpu_lloyd_iters} updates")
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload} (bounded sample)", "precision": "fp64",
                   "sampling": args.sampling},
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
    ap.add_argument("--precision", default="bf16x3", choices=["fp32", "bf16", "bf16x3"])
    ap.add_argument("--workload", default="kdd_n1M_d42_k500")
    ap.add_argument("--sampling", default="bernoulli", choices=["bernoulli", "exact"],
                    help="round draws: independent (Alg. 2 step 4) or exactly l per round (Sec. 5.3)")
    ap.add_argument("--n", type=int, default=0, help="override n (same recipe)")
    ap.add_argument("--ell-factor", type=float, default=0.0, help="override l as a multiple of k")
    ap.add_argument("--cpu-sample-n", type=int, default=40000)
    ap.add_argument("--ref-sample-n", type=int, default=8000)
    ap.add_argument("--cpu-lloyd-iters", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
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
    res = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
