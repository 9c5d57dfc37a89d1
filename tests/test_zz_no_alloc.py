"""kmpar_cost_noalloc: the cost phi_X(C) (Sec. 3.1) for callers that cannot
allocate device memory when they need it (a framework that has reserved all GPU
memory for its own pool, or a latency-critical loop where an allocation, which
can synchronise the device, is not allowed).  Its scratch is a fixed array inside
the library; the result must match kmpar_cost, call after call, and the FP64
oracle's cost.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import math

import numpy as np
import pytest

from paper_1203_6402_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def km():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6402_gb300 import kmpar
    kmpar.load()
    return kmpar


def _case(X, C):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Cd = torch.from_numpy(np.ascontiguousarray(C)).cuda()
    return X, C, Xd, Cd, X.shape[0], X.shape[1], C.shape[0]


def test_noalloc_cost_matches_cost_on_consecutive_calls(km, orc):
    X1 = datagen.kdd_like(20000, seed=31)
    X2 = datagen.gauss_mixture(5003, 15, 8, 10.0, seed=32)
    cases = [_case(X1, X1[::400][:50]), _case(X2, X2[:8])]
    # two calls in a row on each input, and the inputs alternate, so every call
    # reuses the scratch the previous call left behind.  Both entry points run the
    # same kernels in the same order, so the sums are bit-identical.
    for _ in range(2):
        for X, C, Xd, Cd, n, d, k in cases:
            ref = km.kmpar_cost(Xd.data_ptr(), n, d, Cd.data_ptr(), k)
            got = km.kmpar_cost_noalloc(Xd.data_ptr(), n, d, Cd.data_ptr(), k)
            assert got == ref, (got, ref)
            # and against the FP64 definition (FP32 distances: (d+1) 2^-24 relative each)
            assert math.isclose(got, orc.cost(X, C), rel_tol=1e-5)


def test_noalloc_cost_at_its_size_limit(km):
    # n = 8,388,608 = 65,536 blocks of 128 points: every partial slot of the array
    # is written; the previous call (a smaller n) left fewer slots in use
    n, d = 8_388_608, 1
    rng = np.random.Generator(np.random.PCG64(5))
    X = rng.uniform(-1.0, 1.0, size=(n, d)).astype(np.float32)
    C = np.array([[-0.5], [0.25], [0.75]], np.float32)
    Xd = torch.from_numpy(X).cuda()
    Cd = torch.from_numpy(C).cuda()
    for nn in (1000, n, n):
        ref = km.kmpar_cost(Xd.data_ptr(), nn, d, Cd.data_ptr(), 3)
        got = km.kmpar_cost_noalloc(Xd.data_ptr(), nn, d, Cd.data_ptr(), 3)
        assert got == ref, (nn, got, ref)
    # the same cost from the definition, in FP64 on the host
    x = X[:, 0].astype(np.float64)
    exact = np.minimum(np.minimum((x + 0.5) ** 2, (x - 0.25) ** 2), (x - 0.75) ** 2).sum()
    assert math.isclose(got, exact, rel_tol=1e-6)


def test_noalloc_cost_rejects_sizes_beyond_its_limit(km):
    X = torch.zeros(4, 2, device="cuda")
    with pytest.raises(km.KmparError) as e:
        km.kmpar_cost_noalloc(X.data_ptr(), 8_388_609, 2, X.data_ptr(), 1)
    assert e.value.status == km.KMPAR_ERR_ARG
    assert "8,388,608-point limit" in km.kmpar_last_error(None)
