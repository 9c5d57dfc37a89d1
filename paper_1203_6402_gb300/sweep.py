"""Rounds and oversampling sweep of k-means|| (Sec. 5.3, Fig. 5.2).

Runs kmpar_fit (the whole path on the GPU) on one GAUSSMIXTURE data set for every
(r, l) of a grid and several seeds, and reports the median seed and final costs
and candidate counts.  Sec. 5.3 observes that the cost is poor while r l < k (too
few candidates to recluster into k centers) and improves sharply once r l >= k.

    python -m paper_1203_6402_gb300.sweep --rounds 1 2 3 4 5 6 7 8 --ell-factors 0.5 1 2

prints one JSON line per (r, l) and a markdown table.
"""
from __future__ import annotations

import argparse
import json
import statistics

import numpy as np


def sweep(X, k: int, rounds_list, ell_factors, seeds, max_iter: int = 100, precision: str = "fp32"):
    """Median costs over `seeds` for every (r, l = f k); X is an n x d float32 array."""
    import torch

    from . import kmpar as km
    km.load()
    n, d = X.shape
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    C = torch.empty(k, d, dtype=torch.float32, device="cuda")
    prec = km.PRECISIONS[precision]
    rows = []
    for f in ell_factors:
        for r in rounds_list:
            seed_c, final_c, cands, warn = [], [], [], 0
            for s in seeds:
                g = km.KMeansPar(Xd, k, f * k, r, s, precision=prec)
                for i in range(1, r + 1):
                    g.round(i)
                m = g.weight()
                Cs, st = g.recluster()
                out = g.lloyd(Cs, max_iter, hist=True)
                g.close()
                warn += int(st == km.KMPAR_WARN_FEW_CANDIDATES)
                seed_c.append(out["cost_hist"][0])
                final_c.append(out["final_cost"])
                cands.append(m)
            rows.append(dict(r=r, ell=f * k, ell_over_k=f, r_ell_over_k=r * f, seeds=len(seeds),
                             seed_cost=statistics.median(seed_c), final_cost=statistics.median(final_c),
                             candidates=statistics.median(cands), few_candidates_runs=warn))
    return rows


def table(rows) -> str:
    out = ["| l/k | r | r l/k | candidates | median seed cost | median final cost | runs with m < k |",
           "|---:|---:|---:|---:|---:|---:|---:|"]
    for w in rows:
        out.append(f"| {w['ell_over_k']:g} | {w['r']} | {w['r_ell_over_k']:g} | {w['candidates']:g} | "
                   f"{w['seed_cost']:.4g} | {w['final_cost']:.4g} | {w['few_candidates_runs']} |")
    return "\n".join(out)


def main():
    from . import datagen
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--n", type=int, default=10_000)
    ap.add_argument("--d", type=int, default=15)
    ap.add_argument("--k", type=int, default=50)
    ap.add_argument("--R", type=float, default=10.0, help="variance of the mixture's centers")
    ap.add_argument("--rounds", type=int, nargs="+", default=[1, 2, 3, 4, 5, 6, 7, 8])
    ap.add_argument("--ell-factors", type=float, nargs="+", default=[0.5, 1.0, 2.0])
    ap.add_argument("--seeds", type=int, default=11)
    ap.add_argument("--precision", default="fp32")
    args = ap.parse_args()
    X = datagen.gauss_mixture(args.n, args.d, args.k, args.R, seed=2012)
    rows = sweep(X, args.k, args.rounds, args.ell_factors, list(range(args.seeds)), precision=args.precision)
    for w in rows:
        print(json.dumps(w))
    print(table(rows))


if __name__ == "__main__":
    main()
