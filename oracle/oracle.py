"""FP64 CPU oracle for k-means|| -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It loads ``kmpar_oracle.c`` (compiled with
gcc, ``-ffp-contract=off``) through ctypes and chains its step functions in the
order of Algorithm 2 of Bahmani et al., "Scalable K-Means++" (Sec. 3.3):

    init (steps 1-2) -> r rounds of sample (step 4) + union/update (step 5)
    -> weights (step 7) -> weighted k-means++ recluster (step 8, Sec. 4.2)
    -> seed cost (Sec. 3.1) -> Lloyd's iteration (Sec. 1, Sec. 3.1).

It shares no code with the CUDA library; the only thing both sides use is the
seeded input generator module, which holds none of the method's arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kmpar_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

TAG_INIT, TAG_SAMPLE, TAG_RECLUSTER, TAG_EXACT = 1, 2, 3, 4

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i64, i32, u32, u64, f64 = (ctypes.c_int64, ctypes.c_int, ctypes.c_uint32,
                               ctypes.c_uint64, ctypes.c_double)
    sig = {
        "orc_philox4x32_10": (None, [P, P, P]),
        "orc_uniform": (f64, [u64, u32, u32, u64]),
        "orc_dist2_ff": (f64, [P, P, i32]),
        "orc_assign": (f64, [P, i64, i32, P, i64, P, P, P]),
        "orc_cost": (f64, [P, i64, i32, P, i64]),
        "orc_init_index": (i64, [i64, u64]),
        "orc_init": (f64, [P, i64, i32, i64, P, P]),
        "orc_sample": (i64, [P, i64, f64, f64, u32, u64, P, i64, P, P]),
        "orc_sample_exact": (i64, [P, i64, f64, u32, u64, f64, P, P]),
        "orc_update": (f64, [P, i64, i32, P, i64, i64, P, P, P]),
        "orc_weights": (None, [P, i64, i64, P]),
        "orc_recluster": (i32, [P, P, i64, i32, i64, u64, P, P]),
        "orc_recluster_rejection": (i32, [P, P, i64, i32, i64, i64, u64, P, P, P]),
        "orc_lloyd": (i64, [P, i64, i32, P, i64, i64, P, P, P, P]),
        "orc_weighted_lloyd": (i64, [P, P, i64, i32, P, i64, i64, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float32)
    if X.ndim != 2:
        raise ValueError("X must be n x d")
    return X


# ------------------------------------------------------------------ primitives
def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for a 4-word counter and a 2-word key (SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def uniform(i: int, rnd: int, tag: int, seed: int) -> float:
    return _load().orc_uniform(i, rnd, tag, seed)


def assign(X, C):
    """Sec. 3.1: nearest center (lowest index on ties), its d^2, near-tie flags, phi."""
    X = _f32(X)
    C = np.ascontiguousarray(C, dtype=np.float64)
    n, d = X.shape
    k = C.shape[0]
    lab = np.empty(n, np.int64)
    d2 = np.empty(n, np.float64)
    near = np.empty(n, np.int8)
    phi = _load().orc_assign(_p(X), n, d, _p(C), k, _p(lab), _p(d2), _p(near))
    return lab, d2, near.astype(bool), phi


def cost(X, C) -> float:
    """Sec. 3.1: phi_X(C) = sum_x min_i ||x - c_i||^2."""
    X = _f32(X)
    C = np.ascontiguousarray(C, dtype=np.float64)
    return _load().orc_cost(_p(X), X.shape[0], X.shape[1], _p(C), C.shape[0])


def init_index(n: int, seed: int) -> int:
    return _load().orc_init_index(n, seed)


def init(X, i0: int):
    """Algorithm 2 steps 1-2: D^2 to x_i0, idx = 0, psi."""
    X = _f32(X)
    n, d = X.shape
    D2 = np.empty(n, np.float64)
    idx = np.empty(n, np.int64)
    psi = _load().orc_init(_p(X), n, d, i0, _p(D2), _p(idx))
    return D2, idx, psi


def sample(D2, phi: float, ell: float, rnd: int, seed: int):
    """Algorithm 2 step 4: independent draws with p = min(1, l D^2 / phi)."""
    D2 = np.ascontiguousarray(D2, dtype=np.float64)
    n = D2.shape[0]
    out = np.empty(max(n, 1), np.int64)
    p = np.empty(n, np.float64)
    near = np.empty(n, np.int8)
    cnt = _load().orc_sample(_p(D2), n, phi, ell, rnd, seed, _p(out), n, _p(p), _p(near))
    return out[:cnt].copy(), p, near.astype(bool)


def sample_exact(D2, ell: float, rnd: int, seed: int, w: float = 0.0):
    """Sec. 5.3 variant of step 4: exactly floor(l) draws without replacement,
    proportional to D^2 (the earliest exponential clocks -ln(u)/D^2).  Returns the
    drawn points (ascending) and whether another clock rings within w (relative)
    of the last drawn one."""
    D2 = np.ascontiguousarray(D2, dtype=np.float64)
    n = D2.shape[0]
    out = np.empty(max(n, 1), np.int64)
    near = ctypes.c_int8(0)
    cnt = _load().orc_sample_exact(_p(D2), n, ell, rnd, seed, w, _p(out), ctypes.byref(near))
    if cnt < 0:
        raise MemoryError("oracle: out of host memory")
    return out[:cnt].copy(), bool(near.value)


def update(X, sel, first_id: int, D2, idx):
    """Algorithm 2 step 5: union with the rows sel of X; D^2/idx updated in place."""
    X = _f32(X)
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    n, d = X.shape
    near = np.empty(n, np.int8)
    phi = _load().orc_update(_p(X), n, d, _p(sel), sel.shape[0], first_id, _p(D2), _p(idx), _p(near))
    return phi, near.astype(bool)


def weights(idx, m: int) -> np.ndarray:
    """Algorithm 2 step 7."""
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    w = np.empty(max(m, 1), np.int64)
    _load().orc_weights(_p(idx), idx.shape[0], m, _p(w))
    return w[:m].copy()


def recluster(cand, w, k: int, seed: int):
    """Algorithm 2 step 8: weighted k-means++ (Algorithm 1 with multiplicities)."""
    cand = np.ascontiguousarray(cand, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.int64)
    m, d = cand.shape
    chosen = np.empty(k, np.int64)
    near = np.empty(k, np.int8)
    warn = _load().orc_recluster(_p(cand), _p(w), m, d, k, seed, _p(chosen), _p(near))
    return chosen, near.astype(bool), bool(warn)


def recluster_rejection(cand, w, k: int, seed: int, batch: int):
    """Algorithm 2 step 8, the same weighted k-means++ law drawn in batches: up to
    `batch` draws per D^2 snapshot, from 2 batch proposals accepted by rejection.
    Returns (chosen, near, warn, snapshots)."""
    cand = np.ascontiguousarray(cand, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.int64)
    m, d = cand.shape
    chosen = np.empty(k, np.int64)
    near = np.empty(k, np.int8)
    snaps = ctypes.c_int64(0)
    warn = _load().orc_recluster_rejection(_p(cand), _p(w), m, d, k, batch, seed, _p(chosen), _p(near),
                                           ctypes.byref(snaps))
    return chosen, near.astype(bool), bool(warn), int(snaps.value)


def lloyd(X, C, max_iter: int):
    """Lloyd's iteration from centers C (FP64 copy); returns the final state."""
    X = _f32(X)
    C = np.array(C, dtype=np.float64, copy=True, order="C")
    n, d = X.shape
    k = C.shape[0]
    labels = np.empty(n, np.int64)
    fc = ctypes.c_double(0.0)
    hist = np.zeros(max_iter + 1, np.float64)
    near = np.empty(n, np.int8)
    it = _load().orc_lloyd(_p(X), n, d, _p(C), k, max_iter, _p(labels),
                           ctypes.byref(fc), _p(hist), _p(near))
    return C, labels, int(it), fc.value, hist[: it + 1].copy(), near.astype(bool)


# ------------------------------------------------------------------ the chain
@dataclass
class RoundState:
    sel: np.ndarray          # rows of X drawn this round, ascending
    p: np.ndarray            # p_x used for the draw (None for exactly-l rounds)
    near_sample: np.ndarray  # |u - p| <= 1e-6 (exactly-l rounds: the boundary flag)
    D2: np.ndarray           # after the union/update
    idx: np.ndarray
    phi: float
    near_argmin: np.ndarray


@dataclass
class KMeansParResult:
    i0: int
    psi: float
    D2_init: np.ndarray
    rounds: list = field(default_factory=list)
    cand: np.ndarray = None       # candidate row numbers in insertion order
    D2: np.ndarray = None
    idx: np.ndarray = None
    w: np.ndarray = None
    chosen: np.ndarray = None
    recluster_near: np.ndarray = None
    recluster_warn: bool = False
    seed_centers: np.ndarray = None
    seed_cost: float = 0.0


def weighted_lloyd(cand_rows, w, C, max_iter: int):
    """Lloyd's iteration on the weighted candidates (step 8 alternative, Sec. 3.3):
    returns (centers FP64, labels, updates, weighted cost)."""
    cand_rows = _f32(cand_rows)
    w = np.ascontiguousarray(w, dtype=np.int64)
    C = np.array(C, dtype=np.float64, copy=True, order="C")
    m, d = cand_rows.shape
    labels = np.empty(m, np.int64)
    wc = ctypes.c_double(0.0)
    it = _load().orc_weighted_lloyd(_p(cand_rows), _p(w), m, d, _p(C), C.shape[0], max_iter, _p(labels),
                                    ctypes.byref(wc))
    return C, labels, int(it), wc.value


def kmeans_par(X, k: int, ell: float, rounds: int, seed: int, sampling: str = "bernoulli",
               w: float = 0.0, recluster_batch: int = 0) -> KMeansParResult:
    """Algorithm 2 steps 1-8, with per-round snapshots.  sampling="exact" draws
    exactly floor(l) points per round without replacement (Sec. 5.3); w is the
    relative window of its boundary flag.  recluster_batch > 0 draws step 8 in
    batches of that size by rejection (recluster_rejection), else one at a time."""
    X = _f32(X)
    n = X.shape[0]
    i0 = init_index(n, seed)
    D2, idx, psi = init(X, i0)
    res = KMeansParResult(i0=i0, psi=psi, D2_init=D2.copy())
    cand = [i0]
    phi = psi
    for r in range(1, rounds + 1):
        if sampling == "exact":
            sel, bnear = sample_exact(D2, ell, r, seed, w)
            p, nsamp = None, np.array([bnear])
        else:
            sel, p, nsamp = sample(D2, phi, ell, r, seed)
        phi, narg = update(X, sel, len(cand), D2, idx)
        cand.extend(int(s) for s in sel)
        res.rounds.append(RoundState(sel, p, nsamp, D2.copy(), idx.copy(), phi, narg))
    res.cand = np.array(cand, dtype=np.int64)
    res.D2, res.idx = D2, idx
    res.w = weights(idx, len(cand))
    candX = X[res.cand].astype(np.float64)
    if recluster_batch > 0:
        res.chosen, res.recluster_near, res.recluster_warn, _ = recluster_rejection(candX, res.w, k, seed,
                                                                                    recluster_batch)
    else:
        res.chosen, res.recluster_near, res.recluster_warn = recluster(candX, res.w, k, seed)
    res.seed_centers = candX[res.chosen]
    res.seed_cost = cost(X, res.seed_centers)
    return res


def fit(X, k: int, ell: float, rounds: int, seed: int, max_iter: int, sampling: str = "bernoulli",
        recluster_batch: int = 0):
    """k-means|| seeding followed by Lloyd's iteration."""
    par = kmeans_par(X, k, ell, rounds, seed, sampling, recluster_batch=recluster_batch)
    C, labels, it, fc, hist, near = lloyd(X, par.seed_centers, max_iter)
    return par, dict(centers=C, labels=labels, iters=it, final_cost=fc, cost_hist=hist, near=near)
