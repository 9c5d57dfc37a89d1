"""Thin ctypes binding of ``libkmpar.so`` (include/kmpar.h): argument marshalling
only.  Every step of k-means|| runs in the library's CUDA kernels; there is no
Python or CPU fallback -- if the library is missing, loading fails loudly.

The ``kmpar_*`` functions take raw pointers (Python ints: ``tensor.data_ptr()``)
and raise ``KmparError`` on any status other than OK (and the warning, which is
returned).  ``KMeansPar`` wraps a context over a torch CUDA tensor.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libkmpar.so")

KMPAR_OK, KMPAR_ERR_ARG, KMPAR_ERR_CUDA, KMPAR_ERR_OOM, KMPAR_ERR_CAPACITY = 0, 1, 2, 3, 4
KMPAR_ERR_TIMEOUT, KMPAR_ERR_STATE, KMPAR_WARN_FEW_CANDIDATES, KMPAR_ERR_UNSUPPORTED = 5, 6, 7, 8
KMPAR_FP32, KMPAR_BF16, KMPAR_BF16X3, KMPAR_FP8E4M3 = 0, 1, 2, 3
KMPAR_HOST_BUFFERS, KMPAR_EXACT_SAMPLING = 1, 2
KMPAR_SAMPLE_BERNOULLI, KMPAR_SAMPLE_EXACT = 0, 1
SAMPLINGS = {"bernoulli": KMPAR_SAMPLE_BERNOULLI, "exact": KMPAR_SAMPLE_EXACT}
PRECISIONS = {"fp32": KMPAR_FP32, "bf16": KMPAR_BF16, "bf16x3": KMPAR_BF16X3, "fp8": KMPAR_FP8E4M3}

EXPORTED = ["kmpar_init", "kmpar_round", "kmpar_weight", "kmpar_recluster", "kmpar_lloyd", "kmpar_cost",
            "kmpar_fit", "kmpar_state", "kmpar_get_stats", "kmpar_uniforms", "kmpar_set_timing",
            "kmpar_launch_count", "kmpar_cost_noalloc", "kmpar_destroy", "kmpar_release_cached_memory",
            "kmpar_set_sampling", "kmpar_batch_run", "kmpar_batch_cand_capacity", "kmpar_weighted_lloyd",
            "kmpar_batch_set_split", "kmpar_set_recluster",
            "kmpar_status_string", "kmpar_last_error"]


class kmpar_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64),
                ("d", ctypes.c_int32), ("k", ctypes.c_int32), ("rounds_done", ctypes.c_int32),
                ("lloyd_iters", ctypes.c_int32),
                ("round_added", ctypes.c_int64 * 64), ("phi", ctypes.c_double * 65),
                ("sample_near", ctypes.c_int64), ("sample_refined", ctypes.c_int64),
                ("argmin_fp64", ctypes.c_int64), ("argmin_wide", ctypes.c_int64),
                ("recluster_near", ctypes.c_int64),
                ("capacity_overflow", ctypes.c_int32), ("recluster_warn", ctypes.c_int32),
                ("kernel_ms", ctypes.c_double * 2), ("kernel_launches", ctypes.c_int64 * 2),
                ("screen_rows", ctypes.c_int64), ("screen_fallback", ctypes.c_int64),
                ("screen_exact", ctypes.c_int64), ("screen_listed", ctypes.c_int64),
                ("recluster_snapshots", ctypes.c_int64), ("lloyd_settled", ctypes.c_int64)]

    def to_dict(self) -> dict:
        r = self.rounds_done
        return dict(n=self.n, m=self.m, d=self.d, k=self.k, rounds_done=r, lloyd_iters=self.lloyd_iters,
                    round_added=list(self.round_added[:r]), phi=list(self.phi[: r + 1]),
                    sample_near=self.sample_near, sample_refined=self.sample_refined,
                    argmin_fp64=self.argmin_fp64, argmin_wide=self.argmin_wide,
                    recluster_near=self.recluster_near, capacity_overflow=self.capacity_overflow,
                    recluster_warn=self.recluster_warn, kernel_ms=list(self.kernel_ms),
                    kernel_launches=list(self.kernel_launches), screen_rows=self.screen_rows,
                    screen_fallback=self.screen_fallback, screen_exact=self.screen_exact,
                    screen_listed=self.screen_listed, recluster_snapshots=self.recluster_snapshots,
                    lloyd_settled=self.lloyd_settled)


class kmpar_problem(ctypes.Structure):
    _fields_ = [("x_offset", ctypes.c_int64), ("n", ctypes.c_int64), ("d", ctypes.c_int32), ("k", ctypes.c_int32),
                ("ell", ctypes.c_double), ("rounds", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("c_offset", ctypes.c_int64), ("l_offset", ctypes.c_int64),
                ("cand_offset", ctypes.c_int64)]


class kmpar_problem_result(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("seed_cost", ctypes.c_double), ("final_cost", ctypes.c_double),
                ("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("sample_near", ctypes.c_int64),
                ("argmin_fp64", ctypes.c_int64), ("recluster_near", ctypes.c_int64)]

    def to_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class KmparError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"kmpar status {status}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libkmpar.so (built by ``paper_1203_6402_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: run __graft_entry__.build() (nvcc, sm_103a) first")
    lib = ctypes.CDLL(path)
    P, i32, i64, u32, u64, f64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                  ctypes.c_uint64, ctypes.c_double)
    PP = ctypes.POINTER(ctypes.c_void_p)
    sigs = {
        "kmpar_init": (i32, [PP, P, i64, i32, i32, f64, i32, u64, i32, P]),
        "kmpar_round": (i32, [P, i32, ctypes.POINTER(i64), ctypes.POINTER(f64)]),
        "kmpar_weight": (i32, [P, ctypes.POINTER(i64), PP, PP]),
        "kmpar_recluster": (i32, [P, P]),
        "kmpar_lloyd": (i32, [P, P, i32, P, ctypes.POINTER(i32), ctypes.POINTER(f64), P]),
        "kmpar_cost": (i32, [P, i64, i32, P, i32, i32, ctypes.POINTER(f64), P]),
        "kmpar_fit": (i32, [P, i64, i32, i32, f64, i32, u64, i32, i32, P, P, ctypes.POINTER(f64),
                            ctypes.POINTER(f64), ctypes.POINTER(i32), i32, P]),
        "kmpar_state": (i32, [P, PP, PP]),
        "kmpar_get_stats": (i32, [P, ctypes.POINTER(kmpar_stats)]),
        "kmpar_uniforms": (i32, [i64, u32, u32, u64, P, P]),
        "kmpar_set_timing": (i32, [P, i32]),
        "kmpar_set_sampling": (i32, [P, i32]),
        "kmpar_set_recluster": (i32, [P, i32]),
        "kmpar_launch_count": (i64, []),
        "kmpar_cost_noalloc": (i32, [P, i64, i32, P, i32, ctypes.POINTER(f64), P]),
        "kmpar_batch_cand_capacity": (i64, [f64, i32]),
        "kmpar_batch_set_split": (i32, [i32]),
        "kmpar_weighted_lloyd": (i32, [P, P, i32, ctypes.POINTER(i32)]),
        "kmpar_batch_run": (i32, [P, ctypes.POINTER(kmpar_problem), i32, P, P, P, P,
                                  ctypes.POINTER(kmpar_problem_result), P]),
        "kmpar_destroy": (None, [P]),
        "kmpar_release_cached_memory": (i32, []),
        "kmpar_status_string": (ctypes.c_char_p, [i32]),
        "kmpar_last_error": (ctypes.c_char_p, [P]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    _lib = lib
    return lib


def _check(status: int, ctx=None) -> int:
    if status in (KMPAR_OK, KMPAR_WARN_FEW_CANDIDATES):
        return status
    msg = load().kmpar_last_error(ctx)
    raise KmparError(status, (msg or b"").decode() or load().kmpar_status_string(status).decode())


# ------------------------------------------------------------------ same-name wrappers
def kmpar_init(X_ptr: int, n: int, d: int, k: int, ell: float, rounds: int, seed: int, precision: int,
               stream: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().kmpar_init(ctypes.byref(h), X_ptr, n, d, k, ell, rounds, seed, precision, stream))
    return h.value


def kmpar_round(ctx: int, i: int, sync: bool = False):
    if not sync:
        _check(load().kmpar_round(ctx, i, None, None), ctx)
        return None
    na, phi = ctypes.c_int64(), ctypes.c_double()
    _check(load().kmpar_round(ctx, i, ctypes.byref(na), ctypes.byref(phi)), ctx)
    return na.value, phi.value


def kmpar_weight(ctx: int):
    m, ci, w = ctypes.c_int64(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(load().kmpar_weight(ctx, ctypes.byref(m), ctypes.byref(ci), ctypes.byref(w)), ctx)
    return m.value, ci.value, w.value


def kmpar_recluster(ctx: int, centers_ptr: int) -> int:
    return _check(load().kmpar_recluster(ctx, centers_ptr), ctx)


def kmpar_weighted_lloyd(ctx: int, centers_ptr: int, max_iter: int) -> int:
    it = ctypes.c_int32()
    _check(load().kmpar_weighted_lloyd(ctx, centers_ptr, max_iter, ctypes.byref(it)), ctx)
    return it.value


def kmpar_lloyd(ctx: int, centers_ptr: int, max_iter: int, labels_ptr: int | None = None, hist: bool = False):
    it, fc = ctypes.c_int32(), ctypes.c_double()
    buf = (ctypes.c_double * (max_iter + 1))() if hist else None
    _check(load().kmpar_lloyd(ctx, centers_ptr, max_iter, labels_ptr, ctypes.byref(it), ctypes.byref(fc),
                              ctypes.cast(buf, ctypes.c_void_p) if hist else None), ctx)
    return it.value, fc.value, (list(buf[: it.value + 1]) if hist else None)


def kmpar_cost(X_ptr: int, n: int, d: int, C_ptr: int, k: int, precision: int = KMPAR_FP32,
               stream: int = 0) -> float:
    phi = ctypes.c_double()
    _check(load().kmpar_cost(X_ptr, n, d, C_ptr, k, precision, ctypes.byref(phi), stream))
    return phi.value


def kmpar_cost_noalloc(X_ptr: int, n: int, d: int, C_ptr: int, k: int, stream: int = 0) -> float:
    """kmpar_cost without any device allocation (fixed in-library scratch, shared by all calls)."""
    phi = ctypes.c_double()
    _check(load().kmpar_cost_noalloc(X_ptr, n, d, C_ptr, k, ctypes.byref(phi), stream))
    return phi.value


def kmpar_fit(X_ptr: int, n: int, d: int, k: int, ell: float, rounds: int, seed: int, precision: int,
              max_iter: int, centers_ptr: int, labels_ptr: int | None, flags: int = 0, stream: int = 0):
    sc, fc, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    st = _check(load().kmpar_fit(X_ptr, n, d, k, ell, rounds, seed, precision, max_iter, centers_ptr,
                                 labels_ptr, ctypes.byref(sc), ctypes.byref(fc), ctypes.byref(it), flags, stream))
    return dict(seed_cost=sc.value, final_cost=fc.value, iters=it.value, status=st)


def kmpar_batch_cand_capacity(ell: float, rounds: int) -> int:
    return load().kmpar_batch_cand_capacity(ell, rounds)


def kmpar_batch_set_split(rows_per_block: int) -> None:
    _check(load().kmpar_batch_set_split(rows_per_block))


def kmpar_batch_run(X_ptr: int, problems: list, centers_ptr: int, labels_ptr: int | None = None,
                    cand_ptr: int | None = None, w_ptr: int | None = None, stream: int = 0):
    """problems: dicts with the kmpar_problem fields; returns (status, per-problem result dicts).
    A per-problem capacity overflow is reported in its result (status 4), not raised."""
    arr = (kmpar_problem * len(problems))()
    for i, p in enumerate(problems):
        for name, _ in kmpar_problem._fields_:
            setattr(arr[i], name, p[name])
    res = (kmpar_problem_result * len(problems))()
    st = load().kmpar_batch_run(X_ptr, arr, len(problems), centers_ptr, labels_ptr, cand_ptr, w_ptr, res, stream)
    if st not in (KMPAR_OK, KMPAR_WARN_FEW_CANDIDATES, KMPAR_ERR_CAPACITY):
        _check(st)
    return st, [r.to_dict() for r in res]


def kmpar_state(ctx: int):
    d2, idx = ctypes.c_void_p(), ctypes.c_void_p()
    _check(load().kmpar_state(ctx, ctypes.byref(d2), ctypes.byref(idx)), ctx)
    return d2.value, idx.value


def kmpar_get_stats(ctx: int) -> dict:
    s = kmpar_stats()
    _check(load().kmpar_get_stats(ctx, ctypes.byref(s)), ctx)
    return s.to_dict()


def kmpar_uniforms(count: int, rnd: int, tag: int, seed: int, out_ptr: int, stream: int = 0) -> None:
    _check(load().kmpar_uniforms(count, rnd, tag, seed, out_ptr, stream))


def kmpar_set_timing(ctx: int, enable: bool) -> None:
    _check(load().kmpar_set_timing(ctx, 1 if enable else 0), ctx)


def kmpar_set_sampling(ctx: int, mode: int) -> None:
    _check(load().kmpar_set_sampling(ctx, mode), ctx)


def kmpar_set_recluster(ctx: int, batch: int) -> None:
    _check(load().kmpar_set_recluster(ctx, batch), ctx)


def kmpar_launch_count() -> int:
    return load().kmpar_launch_count()


def kmpar_destroy(ctx: int) -> None:
    load().kmpar_destroy(ctx)


def kmpar_release_cached_memory() -> None:
    _check(load().kmpar_release_cached_memory())


# ------------------------------------------------------------------ torch convenience
class KMeansPar:
    """A k-means|| context over a CUDA float32 tensor X (n x d), borrowed."""

    def __init__(self, X, k: int, ell: float, rounds: int, seed: int, precision: str | int = "fp32",
                 stream=None, sampling: str | int = "bernoulli", recluster_batch: int = 0):
        import torch
        if not (X.is_cuda and X.dtype == torch.float32 and X.dim() == 2 and X.is_contiguous()):
            raise ValueError("X must be a contiguous CUDA float32 n x d tensor")
        self.X, self.k = X, k
        self.n, self.d = X.shape
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else precision
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = kmpar_init(X.data_ptr(), self.n, self.d, k, ell, rounds, seed, self.precision,
                              self.stream.cuda_stream)
        self.rounds = rounds
        mode = SAMPLINGS[sampling] if isinstance(sampling, str) else sampling
        try:
            if mode != KMPAR_SAMPLE_BERNOULLI:
                kmpar_set_sampling(self.ctx, mode)
            if recluster_batch:
                kmpar_set_recluster(self.ctx, recluster_batch)
        except KmparError:
            kmpar_destroy(self.ctx)
            self.ctx = None
            raise

    def round(self, i: int, sync: bool = False):
        return kmpar_round(self.ctx, i, sync)

    def weight(self):
        import torch
        m, ci, w = kmpar_weight(self.ctx)
        return m

    def state(self):
        """Copies of D^2 (float32) and idx (int32) as torch tensors."""
        import torch
        d2p, idxp = kmpar_state(self.ctx)
        D2 = torch.empty(self.n, dtype=torch.float32, device=self.X.device)
        idx = torch.empty(self.n, dtype=torch.int32, device=self.X.device)
        _copy_dev(D2.data_ptr(), d2p, 4 * self.n, self.stream)
        _copy_dev(idx.data_ptr(), idxp, 4 * self.n, self.stream)
        return D2, idx

    def candidates(self):
        """(row numbers int32, weights int64) of the candidate set as torch tensors."""
        import torch
        m, ci, w = kmpar_weight(self.ctx)
        cand = torch.empty(m, dtype=torch.int32, device=self.X.device)
        wt = torch.empty(m, dtype=torch.int64, device=self.X.device)
        _copy_dev(cand.data_ptr(), ci, 4 * m, self.stream)
        _copy_dev(wt.data_ptr(), w, 8 * m, self.stream)
        return cand, wt

    def recluster(self):
        import torch
        C = torch.empty(self.k, self.d, dtype=torch.float32, device=self.X.device)
        st = kmpar_recluster(self.ctx, C.data_ptr())
        return C, st

    def lloyd(self, C, max_iter: int, labels: bool = True, hist: bool = False):
        import torch
        lab = torch.empty(self.n, dtype=torch.int32, device=self.X.device) if labels else None
        it, fc, h = kmpar_lloyd(self.ctx, C.data_ptr(), max_iter, lab.data_ptr() if labels else None, hist)
        return dict(labels=lab, iters=it, final_cost=fc, cost_hist=h)

    def stats(self) -> dict:
        return kmpar_get_stats(self.ctx)

    def close(self):
        if self.ctx:
            kmpar_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _copy_dev(dst: int, src: int, nbytes: int, stream) -> None:
    import torch
    if nbytes == 0:
        return
    # a device-to-device byte copy on the given stream through torch (memory plumbing only)
    s = torch.cuda.ExternalStream(stream.cuda_stream) if not isinstance(stream, torch.cuda.Stream) else stream
    with torch.cuda.stream(s):
        src_t = _raw_tensor(src, nbytes)
        dst_t = _raw_tensor(dst, nbytes)
        dst_t.copy_(src_t)


def _raw_tensor(ptr: int, nbytes: int):
    """A uint8 CUDA tensor view of nbytes at ptr (no copy, no ownership)."""
    import torch

    class _Arr:
        def __init__(self, p, nb):
            self.__cuda_array_interface__ = {"shape": (nb,), "typestr": "|u1", "data": (p, False), "version": 3,
                                             "strides": None}

    return torch.as_tensor(_Arr(ptr, nbytes), device="cuda")


def kmpar_status_string(status: int) -> str:
    return load().kmpar_status_string(status).decode()


def kmpar_last_error(ctx: int | None = None) -> str:
    return (load().kmpar_last_error(ctx) or b"").decode()
