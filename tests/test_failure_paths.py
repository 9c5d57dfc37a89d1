"""Error paths of the C ABI, made to happen on the host (failure detection
without a GPU fault): a round that draws more than its capacity (KMPAR_ERR_CAPACITY), a
context whose allocations pass a memory limit (KMPAR_ERR_OOM), and a grid
barrier of the cooperative reclustering kernel whose wait budget runs out
(KMPAR_ERR_TIMEOUT).  No GPU fault is involved: the capacity check, the memory
limit and the bounded wait are the library's own, and after each error the
context (or a new one) still gives the normal result."""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _seed_centers(km, Xd, k, ell, rounds, seed):
    g = km.KMeansPar(Xd, k, ell, rounds, seed)
    for r in range(1, rounds + 1):
        g.round(r)
    g.weight()
    C, _ = g.recluster()
    out = C.cpu().numpy()
    g.close()
    return out


def test_round_capacity_overflow_is_reported(km, monkeypatch):
    Xd = _dev(datagen.gauss_mixture(5000, 8, 10, 10.0, seed=1))
    monkeypatch.setenv("KMPAR_ROUND_CAPACITY", "4")
    g = km.KMeansPar(Xd, 10, 100.0, 3, 2)
    with pytest.raises(km.KmparError) as e:
        g.round(1, sync=True)
    assert e.value.status == km.KMPAR_ERR_CAPACITY
    assert g.stats()["capacity_overflow"] == 1
    g.close()
    # a context made without the override runs the round normally
    monkeypatch.delenv("KMPAR_ROUND_CAPACITY")
    g = km.KMeansPar(Xd, 10, 100.0, 3, 2)
    na, phi = g.round(1, sync=True)
    assert na > 4 and phi > 0
    g.close()


def test_allocation_beyond_the_limit_is_out_of_memory(km, monkeypatch):
    X = datagen.gauss_mixture(20000, 15, 10, 10.0, seed=3)
    Xd = _dev(X)
    monkeypatch.setenv("KMPAR_CTX_LIMIT_BYTES", "100000")
    with pytest.raises(km.KmparError) as e:
        km.KMeansPar(Xd, 10, 20.0, 3, 4)
    assert e.value.status == km.KMPAR_ERR_OOM
    monkeypatch.delenv("KMPAR_CTX_LIMIT_BYTES")
    ref = _seed_centers(km, Xd, 10, 20.0, 3, 4)
    # Lloyd's buffers are allocated by the first kmpar_lloyd: refused there, they are
    # allocated by the next call, which gives the normal result
    g = km.KMeansPar(Xd, 10, 20.0, 3, 4)
    for r in range(1, 4):
        g.round(r)
    g.weight()
    C, _ = g.recluster()
    assert np.array_equal(C.cpu().numpy(), ref)
    C1 = C.clone()
    monkeypatch.setenv("KMPAR_CTX_LIMIT_BYTES", "1")
    with pytest.raises(km.KmparError) as e:
        g.lloyd(C, 20)
    assert e.value.status == km.KMPAR_ERR_OOM
    monkeypatch.delenv("KMPAR_CTX_LIMIT_BYTES")
    out = g.lloyd(C1, 20)
    g.close()
    g2 = km.KMeansPar(Xd, 10, 20.0, 3, 4)
    for r in range(1, 4):
        g2.round(r)
    g2.weight()
    C2, _ = g2.recluster()
    out2 = g2.lloyd(C2, 20)
    g2.close()
    assert out["final_cost"] == out2["final_cost"] and out["iters"] == out2["iters"]


def test_grid_barrier_timeout_returns_an_error_and_the_context_recovers(km, monkeypatch):
    X = datagen.gauss_mixture(20000, 16, 40, 10.0, seed=5)
    Xd = _dev(X)
    monkeypatch.setenv("KMPAR_RECLUSTER_GRID", "1")
    ref = _seed_centers(km, Xd, 40, 200.0, 5, 6)
    g = km.KMeansPar(Xd, 40, 200.0, 5, 6)
    for r in range(1, 6):
        g.round(r)
    m = g.weight()
    assert m > 64          # enough 32-candidate chunks for a grid of several CTAs
    # a one-cycle budget: the first CTA to wait at a barrier gives up at once
    monkeypatch.setenv("KMPAR_WAIT_CYCLES", "1")
    C = torch.empty(40, 16, dtype=torch.float32, device="cuda")
    with pytest.raises(km.KmparError) as e:
        km.kmpar_recluster(g.ctx, C.data_ptr())
    assert e.value.status == km.KMPAR_ERR_TIMEOUT
    assert "timed out" in km.kmpar_last_error(g.ctx)
    # the same context, with the default budget: the normal draws
    monkeypatch.delenv("KMPAR_WAIT_CYCLES")
    C2, st = g.recluster()
    assert np.array_equal(C2.cpu().numpy(), ref)
    out = g.lloyd(C2, 10)
    assert out["iters"] >= 1
    g.close()
