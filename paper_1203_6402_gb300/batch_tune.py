"""Autotuner of the batched path's schedule (kmpar_batch_run).

The one schedule choice of kmpar_batch_run is the size above which a problem is
split over a thread-block cluster (kmpar_batch_set_split).  This script times
kmpar_batch_run on a seeded subset of the batched recipe for each candidate
threshold and writes the fastest to batch_tuning.json beside it, with every
measurement; bench.py applies the table when it exists.

    python -m paper_1203_6402_gb300.batch_tune [--count 1024] [--reps 3]
"""
from __future__ import annotations

import argparse
import json
import os

CANDIDATES = [0, 50_000, 25_000, 12_500, 6_250]
TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch_tuning.json")


def load_table(path: str = TABLE):
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def tune(count: int = 1024, reps: int = 3, seed: int = 4242, candidates=CANDIDATES) -> dict:
    import torch

    from . import datagen
    from . import kmpar as km
    km.load()
    probs = datagen.batched_problems(count, seed=seed)
    X = torch.from_numpy(datagen.batched_points(probs)).cuda()
    C = torch.empty(sum(p["k"] * p["d"] for p in probs), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    times = {}
    for rpb in candidates:
        km.kmpar_batch_set_split(rpb)
        km.kmpar_batch_run(X.data_ptr(), probs, C.data_ptr(), stream=stream.cuda_stream)   # warm-up
        best = float("inf")
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            km.kmpar_batch_run(X.data_ptr(), probs, C.data_ptr(), stream=stream.cuda_stream)
            b.record(stream)
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        times[str(rpb)] = best
    pick = min(candidates, key=lambda r: times[str(r)])
    km.kmpar_batch_set_split(pick)
    return {"rows_per_block": pick, "ms": times, "count": count, "seed": seed,
            "gpu": torch.cuda.get_device_name(0), "note": "0 = never split a problem over a cluster"}


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--count", type=int, default=1024)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=TABLE)
    args = ap.parse_args()
    res = tune(args.count, args.reps)
    with open(args.out, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
