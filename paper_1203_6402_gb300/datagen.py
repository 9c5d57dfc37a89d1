"""Seeded synthetic inputs shaped like the workloads of "Scalable K-Means++".

This module holds no part of the method's arithmetic: it only draws points.  It
is the one module that both the CUDA path's tests/benchmark and the CPU oracle's
tests read, so that both sides see the same bytes.

* ``gauss_mixture`` -- GAUSSMIXTURE (Sec. 4.1): k centers from a spherical
  Gaussian with mean 0 and variance R per coordinate, then points from unit
  variance Gaussians around centers chosen uniformly (equal weights).
* ``kdd_like`` -- a stand-in with the shape of the 4.8M x 42 KDDCUP1999 data
  (Sec. 4.1; the real data set is not available here): 34 heavy-tailed
  non-negative columns (log-normal, mu = 0, sigma = 2), 8 integer-valued columns
  in [0, 255], and a fraction of rows that are exact copies of other rows.

All draws use numpy's PCG64 with an explicit seed; outputs are FP32, row-major.
"""
from __future__ import annotations

import numpy as np


def gauss_mixture(n: int, d: int, k_true: int, R: float, seed: int, return_centers: bool = False):
    """R is the variance of each center coordinate (centers ~ N(0, R I_d)), the
    reading every workload of this module uses (Sec. 4.1 prints "variance R")."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centers = rng.normal(0.0, np.sqrt(R), size=(k_true, d))
    comp = rng.integers(0, k_true, size=n)
    # the unit-variance offsets are drawn in row blocks: the generator fills values in
    # order, so the points are the same as one draw of n x d, without its FP64 copy
    X = np.empty((n, d), dtype=np.float32)
    block = max(1, (1 << 22) // max(1, d))
    for i in range(0, n, block):
        j = min(n, i + block)
        X[i:j] = (centers[comp[i:j]] + rng.normal(0.0, 1.0, size=(j - i, d))).astype(np.float32)
    if return_centers:
        return X, centers, comp
    return X


def kdd_like(n: int, seed: int, d_lognormal: int = 34, d_int: int = 8, dup_frac: float = 0.2,
             sigma: float = 2.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    d = d_lognormal + d_int
    X = np.empty((n, d), dtype=np.float32)
    X[:, :d_lognormal] = rng.lognormal(0.0, sigma, size=(n, d_lognormal)).astype(np.float32)
    X[:, d_lognormal:] = rng.integers(0, 256, size=(n, d_int)).astype(np.float32)
    ndup = int(round(dup_frac * n))
    if ndup > 0 and n > 1:
        dst = rng.choice(n, size=ndup, replace=False)
        src = rng.integers(0, n, size=ndup)
        X[dst] = X[src]
    return X


def uniform_box(n: int, d: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Plain uniform points (edge-case tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=(n, d)).astype(np.float32)


# The five workloads, by name.  Sizes follow the benchmark table of the design.
WORKLOADS = {
    "gmm_n10k_d15_k50": dict(kind="gmm", n=10_000, d=15, k=50, k_true=50, R=10.0, ell=100.0, rounds=5,
                             max_iter=100),
    "kdd_n1M_d42_k500": dict(kind="kdd", n=1_000_000, d=42, k=500, ell=1000.0, rounds=5, max_iter=100),
    "kdd_n4.8M_d42_k1000": dict(kind="kdd", n=4_800_000, d=42, k=1000, ell=2000.0, rounds=5, max_iter=100),
    "gmm_n10M_d128_k10000": dict(kind="gmm", n=10_000_000, d=128, k=10_000, k_true=10_000, R=100.0,
                                 ell=20_000.0, rounds=5, max_iter=10),
}

# Lloyd caps, stated with each workload: the GAUSSMIXTURE configuration asks for
# convergence within 100 iterations; the 1e7 x 128 one states no cap, and 10 updates
# (the batched configuration's count) keep one step near a second.


def make(name: str, seed: int, n: int | None = None) -> np.ndarray:
    """Points for a named workload (optionally a smaller n with the same recipe)."""
    w = WORKLOADS[name]
    nn = w["n"] if n is None else n
    if w["kind"] == "gmm":
        return gauss_mixture(nn, w["d"], w["k_true"], w["R"], seed)
    return kdd_like(nn, seed)


def batched_problems(count: int, seed: int, n_lo: int = 1_000, n_hi: int = 200_000, k_lo: int = 16,
                     k_hi: int = 256, dims=(32, 64, 128), R: float = 10.0, rounds: int = 5, max_iter: int = 10):
    """Descriptions of `count` independent GAUSSMIXTURE problems: n and k
    log-uniform in [n_lo, n_hi] and [k_lo, k_hi] (k at most n), d uniform over
    `dims`, l = 2k, each with its own data seed and run seed, and the offsets of
    its rows in one concatenated X (row-major, float32), of its k x d centers and
    of its labels."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=count)).astype(np.int64)
    k = np.exp(rng.uniform(np.log(k_lo), np.log(k_hi), size=count)).astype(np.int64)
    k = np.minimum(k, n)
    d = rng.choice(np.asarray(dims), size=count)
    probs = []
    xo = co = lo = 0
    for i in range(count):
        probs.append(dict(x_offset=xo, n=int(n[i]), d=int(d[i]), k=int(k[i]), ell=2.0 * int(k[i]), rounds=rounds,
                          max_iter=max_iter, seed=int(seed) * 100003 + i, data_seed=int(seed) * 7919 + i,
                          c_offset=co, l_offset=lo, cand_offset=0))
        xo += int(n[i]) * int(d[i])
        co += int(k[i]) * int(d[i])
        lo += int(n[i])
    return probs


def batched_points(problems, out=None) -> np.ndarray:
    """The concatenated X of batched_problems (each problem its own mixture of k
    components, centers ~ N(0, R I), unit-variance points), float32."""
    total = sum(p["n"] * p["d"] for p in problems)
    X = np.empty(total, dtype=np.float32) if out is None else out
    for p in problems:
        Xi = gauss_mixture(p["n"], p["d"], p["k"], 10.0, p["data_seed"])
        X[p["x_offset"]: p["x_offset"] + p["n"] * p["d"]] = Xi.ravel()
    return X
