"""GPU parity: every step of k-means|| through the C ABI against the FP64 oracle
on the same seeded inputs (Algorithm 2, Sec. 3.3; Lloyd, Sec. 3.1).

Bar (per step): candidate sets and weights bit-exact; idx/labels bit-exact except
where the oracle reports a near tie (runner-up within 1e-6 relative); draws
bit-exact except where the oracle reports |u - p| <= 1e-6; D^2 within 1e-5
relative (exact FP32 difference form vs FP64; absolute floor 1e-30); phi within
1e-6 relative; final Lloyd cost within 1e-4 relative.
"""
import math

import numpy as np
import pytest

from paper_1203_6402_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D2_RTOL = 1e-5


@pytest.fixture(scope="module")
def km():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6402_gb300 import kmpar
    kmpar.load()
    return kmpar


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _close_d2(gpu, ref):
    ref = np.asarray(ref, np.float64)
    gpu = np.asarray(gpu, np.float64)
    return np.abs(gpu - ref) <= D2_RTOL * np.abs(ref) + 1e-30


def run_and_compare(km, orc, X, k, ell, rounds, seed, precision="fp32", max_iter=100, sampling="bernoulli",
                    recluster_batch=0):
    """Runs the GPU path step by step and the oracle beside it; asserts the bar.

    Returns a dict of diagnostics.  If the trajectories part at a reported near
    tie, the remaining steps are checked for validity only (diag['parted'])."""
    n, d = X.shape
    Xd = _dev(X)
    g = km.KMeansPar(Xd, k, ell, rounds, seed, precision=precision, sampling=sampling,
                     recluster_batch=recluster_batch)
    diag = dict(parted=None, boundary_near=[])
    # exactly-l rounds: the relative window in which FP32 and exact clocks may swap
    wwin = (2 * d + 16) * 2.0 ** -24
    # Alg. 2 steps 1-2
    i0 = orc.init_index(n, seed)
    D2, idx, psi = orc.init(X, i0)
    gD2, gidx = g.state()
    assert np.all(_close_d2(gD2.cpu().numpy(), D2))
    assert np.all(gidx.cpu().numpy() == 0)
    cand = [i0]
    phi = psi
    for r in range(1, rounds + 1):
        if sampling == "exact":
            sel, bnear = orc.sample_exact(D2, ell, r, seed, wwin)
            diag["boundary_near"].append(bnear)
        else:
            sel, p, nsamp = orc.sample(D2, phi, ell, r, seed)
        phi, narg = orc.update(X, sel, len(cand), D2, idx)
        na, gphi = g.round(r, sync=True)
        cand.extend(int(s) for s in sel)
        gD2, gidx = g.state()
        gD2, gidx = gD2.cpu().numpy(), gidx.cpu().numpy()
        if na != len(sel):
            diag["parted"] = ("round", r)
            break
        assert math.isclose(gphi, phi, rel_tol=1e-6), (r, gphi, phi)
        ok_d2 = _close_d2(gD2, D2)
        ok_idx = gidx == idx
        bad = ~(ok_d2 & ok_idx) & ~narg
        assert not bad.any(), f"round {r}: {bad.sum()} points differ (first {np.flatnonzero(bad)[:5]})"
    stats = g.stats()
    diag["stats"] = stats
    m, ci, wp = km.kmpar_weight(g.ctx)
    gcand, gw = g.candidates()
    gcand, gw = gcand.cpu().numpy(), gw.cpu().numpy()
    if diag["parted"] is None:
        if not np.array_equal(gcand, np.array(cand)):
            # a draw may flip only at a reported near tie
            diag["parted"] = ("candidates", None)
        else:
            w = orc.weights(idx, len(cand))
            assert np.array_equal(gw, w)
    assert gw.sum() == n                                             # step 7: sum w = n
    C, st = g.recluster()
    Ch = C.cpu().numpy()
    # the seed centers are rows of X from the candidate set
    rows = gcand
    if diag["parted"] is None:
        if recluster_batch:
            chosen, rnear, rwarn, snaps = orc.recluster_rejection(X[rows].astype(np.float64), gw, k, seed,
                                                                  recluster_batch)
            gst = g.stats()
            if not rnear.any() and gst["recluster_near"] == 0:
                assert gst["recluster_snapshots"] == snaps
            diag["recluster_snapshots"] = gst["recluster_snapshots"]
        else:
            chosen, rnear, rwarn = orc.recluster(X[rows].astype(np.float64), gw, k, seed)
        assert (st == km.KMPAR_WARN_FEW_CANDIDATES) == rwarn
        same = np.all(Ch == X[rows[chosen]], axis=1)
        if not same.all():
            assert rnear.any() or stats["recluster_near"] > 0, "recluster differs without a reported near tie"
            diag["parted"] = ("recluster", int(np.argmin(same)))
    C0 = Ch.copy()
    out = g.lloyd(C, max_iter, labels=True, hist=True)
    Cf = C.cpu().numpy()
    lab = out["labels"].cpu().numpy()
    # Lloyd from the same seed centers in the oracle
    oC, olab, oit, ofc, ohist, onear = orc.lloyd(X, C0.astype(np.float64), max_iter)
    seed_cost = orc.cost(X, C0.astype(np.float64))
    assert math.isclose(out["cost_hist"][0], seed_cost, rel_tol=1e-6)
    if out["iters"] == oit and np.array_equal(lab, olab):
        assert math.isclose(out["final_cost"], ofc, rel_tol=1e-4)
        np.testing.assert_allclose(Cf, oC, rtol=1e-5, atol=1e-5 * (np.abs(oC).max() + 1))
    else:
        # a Lloyd trajectory may part only at a near tie; the final state must still be valid
        assert onear.any() or diag["stats"]["argmin_fp64"] > 0
        diag["lloyd_parted"] = True
        assert out["final_cost"] <= seed_cost * (1 + 1e-6)
    # the GPU's final labels are the nearest centers of its final centers (FP64 check)
    Cf64 = Cf.astype(np.float64)
    D = ((X.astype(np.float64)[:, None, :] - Cf64[None]) ** 2).sum(-1) if n * k <= 4_000_000 else None
    if D is not None:
        best = D.min(1)
        assert np.all(D[np.arange(n), lab] <= best * (1 + 1e-6) + 1e-30)
        assert math.isclose(out["final_cost"], best.sum(), rel_tol=1e-5)
    hist = np.array(out["cost_hist"])
    assert np.all(np.diff(hist) <= 1e-6 * hist[0])                   # cost never increases
    diag["iters"] = out["iters"]
    diag["final_cost"] = out["final_cost"]
    g.close()
    return diag


CASES = [
    # name, X maker, k, ell, rounds, seed
    ("gmm_small", lambda: datagen.gauss_mixture(3000, 15, 20, 10.0, seed=1), 20, 40.0, 5, 3),
    ("kdd_like", lambda: datagen.kdd_like(2500, seed=2), 30, 60.0, 5, 4),
    ("ragged_d1", lambda: datagen.uniform_box(1001, 1, seed=3), 7, 14.0, 4, 5),
    ("d130_generic", lambda: datagen.gauss_mixture(777, 130, 6, 4.0, seed=4), 6, 12.0, 3, 6),
    ("d128", lambda: datagen.gauss_mixture(1500, 128, 12, 100.0, seed=5), 12, 24.0, 5, 7),
    ("d42_many_centers", lambda: datagen.kdd_like(2000, seed=6), 64, 300.0, 3, 8),
    # the GAUSSMIXTURE configuration exactly: n = 10^4, d = 15, 50 centers ~ N(0, 10 I),
    # k = 50, l = 2k, r = 5, Lloyd to convergence within 100 updates
    ("gmm_config_n10k_d15_k50", lambda: datagen.make("gmm_n10k_d15_k50", seed=1000), 50, 100.0, 5, 7),
]


@pytest.mark.parametrize("name,mk,k,ell,rounds,seed", CASES, ids=[c[0] for c in CASES])
def test_parity_fp32(km, orc, name, mk, k, ell, rounds, seed):
    X = mk()
    diag = run_and_compare(km, orc, X, k, ell, rounds, seed)
    assert diag["parted"] is None, diag


TC_CASES = [c for c in CASES if c[0] != "d130_generic"] + [
    ("gmm_d42_multi_tile", lambda: datagen.gauss_mixture(9000, 42, 40, 10.0, seed=13), 300, 600.0, 3, 9),
    ("kdd_ragged_3001", lambda: datagen.kdd_like(3001, seed=14), 40, 80.0, 4, 10),
    # round batches of ~1,500 candidates: the resident refine runs in three slices
    ("kdd_sliced_batches", lambda: datagen.kdd_like(6000, seed=16), 100, 1500.0, 2, 11),
    # 321 row tiles: every persistent CTA of the screening pass takes two or three A
    # tiles, so the TMEM buffers, the A ring and the L2 prefetch wrap around
    ("kdd_n41k_multi_tile_per_cta", lambda: datagen.kdd_like(41000, seed=17), 50, 100.0, 3, 12),
    # the 1e7 x 128 configuration's shape at 1/500 of its size (1,000 points per
    # cluster, centers ~ N(0, 100 I), l = 2k): a round batch holds several candidates
    # of one cluster, closer together than the BF16/FP8 screening bound, so many rows
    # go through the list pass
    ("gmm_d128_dense_clusters", lambda: datagen.gauss_mixture(20000, 128, 20, 100.0, seed=18), 20, 40.0, 5, 13),
]


@pytest.mark.parametrize("precision", ["bf16x3", "bf16", "fp8"])
@pytest.mark.parametrize("name,mk,k,ell,rounds,seed", TC_CASES, ids=[c[0] for c in TC_CASES])
def test_parity_tensor_screening(km, orc, name, mk, k, ell, rounds, seed, precision):
    """tcgen05 screening + exact refine: same decisions as the oracle (and the FP32 path)."""
    X = mk()
    if precision == "bf16x3" and 3 * X.shape[1] + 4 > 192:
        # split mode carries 3d + 4 K columns; at most three 64-column atoms are built
        with pytest.raises(km.KmparError) as e:
            km.KMeansPar(_dev(X), k, ell, rounds, seed, precision=precision)
        assert e.value.status == km.KMPAR_ERR_UNSUPPORTED
        return
    diag = run_and_compare(km, orc, X, k, ell, rounds, seed, precision=precision)
    assert diag["parted"] is None, diag
    st = diag["stats"]
    assert st["screen_rows"] > 0
    if precision == "bf16x3" and name.startswith("gmm"):
        # well-separated data: nearly every row is decided by the screening alone
        assert st["screen_fallback"] <= 0.05 * st["screen_rows"], st
    assert st["screen_exact"] <= st["screen_fallback"]
    if name == "gmm_d128_dense_clusters":
        # rows left undecided by the pair screening were there, and the list pass
        # settled most of them without the exact scan
        assert st["screen_fallback"] > 0 and st["screen_exact"] < 0.5 * st["screen_fallback"], st


EXACT_CASES = [
    # name, X maker, k, ell, rounds, seed, precision
    ("gmm_small", lambda: datagen.gauss_mixture(3000, 15, 20, 10.0, seed=1), 20, 40.0, 5, 3, "fp32"),
    ("kdd_like", lambda: datagen.kdd_like(2500, seed=2), 30, 60.0, 5, 4, "bf16x3"),
    ("kdd_sliced_batches", lambda: datagen.kdd_like(6000, seed=16), 100, 1500.0, 2, 11, "bf16x3"),
    # 30 drawn, then the 9 points left with D^2 > 0, then none
    ("tiny_all_drawn", lambda: datagen.uniform_box(40, 3, seed=21), 5, 30.0, 3, 6, "fp32"),
]


@pytest.mark.parametrize("name,mk,k,ell,rounds,seed,precision", EXACT_CASES, ids=[c[0] for c in EXACT_CASES])
def test_parity_exact_rounds(km, orc, name, mk, k, ell, rounds, seed, precision):
    """Exactly-l rounds (Sec. 5.3): floor(l) draws per round without replacement,
    proportional to D^2 -- the same draws as the oracle's exponential clocks, then
    the same union, weights, recluster and Lloyd."""
    X = mk()
    diag = run_and_compare(km, orc, X, k, ell, rounds, seed, precision=precision, sampling="exact")
    assert not any(diag["boundary_near"]), diag["boundary_near"]
    assert diag["parted"] is None, diag   # so every round drew what the oracle drew


def test_exact_sampling_arguments(km):
    X = _dev(datagen.uniform_box(100, 2, seed=1))
    g = km.KMeansPar(X, 3, 5.0, 2, 1)
    g.round(1)
    with pytest.raises(km.KmparError) as e:
        km.kmpar_set_sampling(g.ctx, km.KMPAR_SAMPLE_EXACT)
    assert e.value.status == km.KMPAR_ERR_STATE
    g.close()
    with pytest.raises(km.KmparError) as e:
        km.KMeansPar(X, 3, 0.5, 2, 1, sampling="exact")
    assert e.value.status == km.KMPAR_ERR_ARG
    g = km.KMeansPar(X, 3, 5.0, 2, 1)
    with pytest.raises(km.KmparError) as e:
        km.kmpar_set_sampling(g.ctx, 7)
    assert e.value.status == km.KMPAR_ERR_ARG
    g.close()


def test_tensor_paths_match_fp32_path(km):
    X = datagen.kdd_like(20000, seed=15)
    Xd = _dev(X)
    res = {}
    for prec in ("fp32", "bf16x3", "bf16", "fp8"):
        g = km.KMeansPar(Xd, 64, 128.0, 5, 3, precision=prec)
        for r in range(1, 6):
            g.round(r)
        cand, w = g.candidates()
        C, _ = g.recluster()
        out = g.lloyd(C, 20)
        res[prec] = (cand.cpu().numpy(), w.cpu().numpy(), C.cpu().numpy(), out["labels"].cpu().numpy(),
                     out["final_cost"], g.stats())
        g.close()
    for prec in ("bf16x3", "bf16", "fp8"):
        for a, b in zip(res["fp32"][:4], res[prec][:4]):
            assert np.array_equal(a, b), prec
        assert res["fp32"][4] == res[prec][4]


def test_tensor_paths_match_fp32_path_wide_rows(km):
    """d = 128 (BF16 with the norms added in the epilogue, FP8 e4m3): dense
    clusters send rows through the list pass; every decision equals the FP32 path's."""
    X = datagen.gauss_mixture(60000, 128, 60, 100.0, seed=19)
    Xd = _dev(X)
    res = {}
    for prec in ("fp32", "bf16", "fp8"):
        g = km.KMeansPar(Xd, 60, 120.0, 5, 4, precision=prec)
        for r in range(1, 6):
            g.round(r)
        D2, idx = g.state()
        cand, w = g.candidates()
        C, _ = g.recluster()
        out = g.lloyd(C, 10)
        res[prec] = (cand.cpu().numpy(), w.cpu().numpy(), D2.cpu().numpy(), idx.cpu().numpy(), C.cpu().numpy(),
                     out["labels"].cpu().numpy(), out["final_cost"], g.stats())
        g.close()
    for prec in ("bf16", "fp8"):
        for a, b in zip(res["fp32"][:6], res[prec][:6]):
            assert np.array_equal(a, b), prec
        assert res["fp32"][6] == res[prec][6]
        st = res[prec][7]
        assert st["screen_fallback"] > 0 and st["screen_exact"] < st["screen_fallback"], (prec, st)


def test_round_pass_lists_match_fp32_path(km):
    """Round batches too large for the resident refine (d = 128, l = 800): the screening
    takes groups of four and, from the second round on, keeps every row's list of the
    centers within the bound of its D^2 in the screening pass itself; the rows it leaves
    undecided are refined from those lists.  Every round's D^2 and idx, the candidates and
    the weights equal the FP32 path's."""
    X = datagen.gauss_mixture(200000, 128, 400, 100.0, seed=23)
    Xd = _dev(X)
    res = {}
    for prec in ("fp32", "bf16", "fp8"):
        g = km.KMeansPar(Xd, 400, 800.0, 4, 5, precision=prec)
        per = []
        for r in range(1, 5):
            g.round(r)
            D2, idx = g.state()
            per.append((D2.cpu().numpy(), idx.cpu().numpy()))
        cand, w = g.candidates()
        res[prec] = (per, cand.cpu().numpy(), w.cpu().numpy(), g.stats())
        g.close()
    for prec in ("bf16", "fp8"):
        for r, ((a1, b1), (a2, b2)) in enumerate(zip(res["fp32"][0], res[prec][0])):
            assert np.array_equal(a1, a2) and np.array_equal(b1, b2), (prec, r + 1)
        assert np.array_equal(res["fp32"][1], res[prec][1]) and np.array_equal(res["fp32"][2], res[prec][2])
        st = res[prec][3]
        assert 0 < st["screen_listed"] <= st["screen_fallback"], (prec, st)


def test_tensor_precision_rejects_large_d(km):
    # BF16 carries d + 2 K columns, split BF16 3d + 2; three 64-column atoms are built
    X = _dev(datagen.uniform_box(200, 200, seed=1))
    for prec in ("bf16", "bf16x3", "fp8"):
        with pytest.raises(km.KmparError) as e:
            km.KMeansPar(X, 4, 8.0, 2, 0, precision=prec)
        assert e.value.status == km.KMPAR_ERR_UNSUPPORTED


def test_philox_matches_oracle(km, orc):
    for rnd, tag, seed in [(0, 1, 0), (3, 2, 12345), (0, 3, (1 << 40) + 7)]:
        out = torch.empty(20000, dtype=torch.float64, device="cuda")
        km.kmpar_uniforms(20000, rnd, tag, seed, out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = np.array([orc.uniform(i, rnd, tag, seed) for i in range(20000)])
        assert np.array_equal(got, ref)


def test_cost_matches_oracle(km, orc):
    X = datagen.kdd_like(5000, seed=9)
    C = X[::97][:40].copy()
    Xd, Cd = _dev(X), _dev(C)          # keep both alive while the library reads them
    phi = km.kmpar_cost(Xd.data_ptr(), 5000, X.shape[1], Cd.data_ptr(), len(C))
    assert math.isclose(phi, orc.cost(X, C.astype(np.float64)), rel_tol=1e-6)


def test_fit_host_buffers_matches_device(km):
    X = datagen.gauss_mixture(4000, 15, 12, 10.0, seed=11)
    n, d = X.shape
    k = 12
    Xd = _dev(X)
    Cd = torch.empty(k, d, dtype=torch.float32, device="cuda")
    Ld = torch.empty(n, dtype=torch.int32, device="cuda")
    r1 = km.kmpar_fit(Xd.data_ptr(), n, d, k, 24.0, 5, 3, km.KMPAR_FP32, 50, Cd.data_ptr(), Ld.data_ptr())
    Ch = np.zeros((k, d), np.float32)
    Lh = np.zeros(n, np.int32)
    r2 = km.kmpar_fit(X.ctypes.data, n, d, k, 24.0, 5, 3, km.KMPAR_FP32, 50, Ch.ctypes.data, Lh.ctypes.data,
                      flags=km.KMPAR_HOST_BUFFERS)
    assert r1["final_cost"] == r2["final_cost"] and r1["iters"] == r2["iters"]
    assert np.array_equal(Cd.cpu().numpy(), Ch) and np.array_equal(Ld.cpu().numpy(), Lh)


def test_run_to_run_deterministic(km):
    X = datagen.kdd_like(30000, seed=12)
    Xd = _dev(X)
    res = []
    for _ in range(3):
        g = km.KMeansPar(Xd, 50, 100.0, 5, 21)
        for r in range(1, 6):
            g.round(r)
        g.weight()
        C, _ = g.recluster()
        out = g.lloyd(C, 30)
        res.append((C.cpu().numpy(), out["labels"].cpu().numpy(), out["final_cost"]))
        g.close()
        # the second context reuses the pooled buffers of the first; before the
        # third, the pool hands its memory back to the driver
        if len(res) == 2:
            km.kmpar_release_cached_memory()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert np.array_equal(res[0][0], res[2][0]) and np.array_equal(res[0][1], res[2][1])
    assert res[0][2] == res[1][2] == res[2][2]


@pytest.mark.parametrize("form", ["cluster", "grid"])
def test_recluster_forms_match_oracle(km, orc, form, monkeypatch):
    """Weighted k-means++ (Alg. 2 step 8) in both kernel forms: one thread-block
    cluster with distributed shared memory, and the cooperative grid."""
    if form == "grid":
        monkeypatch.setenv("KMPAR_RECLUSTER_GRID", "1")
    X = datagen.kdd_like(6000, seed=41)
    diag = run_and_compare(km, orc, X, 80, 160.0, 5, 17)
    assert diag["parted"] is None, diag


@pytest.mark.parametrize("batch", [1, 4, 64])
def test_recluster_batched_matches_oracle(km, orc, batch):
    """Step 8 drawn in batches by rejection from a D^2 snapshot (the same weighted
    k-means++ law): the chosen rows and the number of snapshots equal the oracle's."""
    X = datagen.kdd_like(6000, seed=41)
    diag = run_and_compare(km, orc, X, 80, 160.0, 5, 17, recluster_batch=batch)
    assert diag["parted"] is None, diag
    assert diag["recluster_snapshots"] >= -(-79 // batch)


def test_set_recluster_validates_and_both_forms_run_on_one_context(km, orc):
    """kmpar_set_recluster: batches outside 0..64 are refused (KMPAR_ERR_ARG); one
    context reclusters in both forms, each equal to its oracle function."""
    X = datagen.gauss_mixture(3000, 8, 12, 10.0, seed=3)
    k, seed = 12, 19
    g = km.KMeansPar(_dev(X), k, 24.0, 3, seed)
    for b in (-1, 65):
        with pytest.raises(km.KmparError) as ei:
            km.kmpar_set_recluster(g.ctx, b)
        assert ei.value.status == km.KMPAR_ERR_ARG
    for r in range(1, 4):
        g.round(r)
    g.weight()
    cand, w = g.candidates()
    cand, w = cand.cpu().numpy(), w.cpu().numpy()
    rows = X[cand].astype(np.float64)
    for b in (0, 5, 0):
        km.kmpar_set_recluster(g.ctx, b)
        C, _ = g.recluster()
        if b:
            ch, near, _, _ = orc.recluster_rejection(rows, w, k, seed, b)
        else:
            ch, near, _ = orc.recluster(rows, w, k, seed)
        if not near.any():
            assert np.array_equal(C.cpu().numpy(), X[cand[ch]]), b
    g.close()


def test_recluster_batched_many_snapshots(km, orc):
    """~20,000 candidates, k = 1,500, 64 draws per snapshot: the reclustering alone
    (on the GPU's own candidate set) against the oracle, draw by draw up to the
    first reported near tie."""
    X = datagen.gauss_mixture(60000, 16, 300, 10.0, seed=5)
    k = 1500
    g = km.KMeansPar(_dev(X), k, 4000.0, 5, 23, recluster_batch=64)
    for r in range(1, 6):
        g.round(r)
    g.weight()
    gcand, gw = g.candidates()
    gcand, gw = gcand.cpu().numpy(), gw.cpu().numpy()
    C, st = g.recluster()
    gst = g.stats()
    g.close()
    assert len(gcand) > 15000
    chosen, rnear, rwarn, snaps = orc.recluster_rejection(X[gcand].astype(np.float64), gw, k, 23, 64)
    assert not rwarn and st == km.KMPAR_OK
    same = np.all(C.cpu().numpy() == X[gcand[chosen]], axis=1)
    # the sequences may part only at a draw the oracle flags (a target or an
    # acceptance test near a boundary); flagged draws mostly still agree
    bad = np.flatnonzero(~same)
    if bad.size:
        assert rnear[: bad[0] + 1].any(), f"draw {bad[0]} differs without a reported near tie"
        assert bad[0] >= 100, f"the sequences part early, at draw {bad[0]}"
    else:
        assert gst["recluster_snapshots"] == snaps
    assert snaps >= -(-(k - 1) // 64)


@pytest.mark.parametrize("k,d,precision", [(420, 128, "fp32"), (37, 15, "fp32"), (1000, 42, "bf16x3")],
                         ids=["many_wide_clusters", "few_narrow_clusters", "sliced_resident_refine"])
def test_lloyd_from_fixed_centers_matches_oracle(km, orc, k, d, precision):
    """Lloyd alone (Sec. 3.1 centroid, Sec. 1 iteration) from fixed seed centers:
    the segmented centroid sums and the assignment agree with the oracle, also
    with many clusters of wide rows (k = 420, d = 128) and with 1,000 centers
    screened on the tensor cores (their refine runs in two shared-memory slices)."""
    X = datagen.gauss_mixture(2500, d, 40, 100.0, seed=33)
    C0 = np.ascontiguousarray(X[:k])
    g = km.KMeansPar(_dev(X), k, 2.0 * k, 1, 5, precision=precision)
    C = _dev(C0)
    out = g.lloyd(C, 15, labels=True, hist=True)
    lab = out["labels"].cpu().numpy()
    oC, olab, oit, ofc, ohist, onear = orc.lloyd(X, C0.astype(np.float64), 15)
    if out["iters"] == oit and np.array_equal(lab, olab):
        assert math.isclose(out["final_cost"], ofc, rel_tol=1e-4)
        oCf = np.asarray(oC)
        np.testing.assert_allclose(C.cpu().numpy(), oCf, rtol=1e-5, atol=1e-5 * (np.abs(oCf).max() + 1))
    else:
        assert onear.any() or g.stats()["argmin_fp64"] > 0
    g.close()


def test_lloyd_bounds_settle_rows_and_match_oracle(km, orc):
    """Lloyd in BF16 at d = 128 (norms in the screening epilogue, direct refine):
    after the first assignment, rows whose bounds (upper bound to their center plus
    its drift below the lower bound to every other center minus their largest drift)
    prove the center unchanged skip the tensor pass.  The trajectory equals the
    oracle's, and the labels and centers equal the FP32 path's bit for bit."""
    X = datagen.gauss_mixture(30000, 128, 60, 100.0, seed=91)
    k = 60
    C0 = np.ascontiguousarray(X[::499][:k])
    res = {}
    for prec in ("bf16", "fp32"):
        g = km.KMeansPar(_dev(X), k, 2.0 * k, 1, 5, precision=prec)
        C = _dev(C0)
        out = g.lloyd(C, 15, labels=True, hist=True)
        res[prec] = (C.cpu().numpy(), out["labels"].cpu().numpy(), out["iters"], out["final_cost"], g.stats())
        g.close()
    Cb, lb, itb, fcb, stb = res["bf16"]
    Cf, lf, itf, fcf, stf = res["fp32"]
    assert stb["lloyd_settled"] > 0 and stf["lloyd_settled"] == 0
    assert itb == itf and np.array_equal(lb, lf) and np.array_equal(Cb, Cf) and fcb == fcf
    oC, olab, oit, ofc, ohist, onear = orc.lloyd(X, C0.astype(np.float64), 15)
    if itb == oit and np.array_equal(lb, olab):
        assert math.isclose(fcb, ofc, rel_tol=1e-4)
        np.testing.assert_allclose(Cb, oC, rtol=1e-5, atol=1e-5 * (np.abs(oC).max() + 1))
    else:
        assert onear.any() or stb["argmin_fp64"] > 0


# ------------------------------------------------------------------ edge cases
def test_single_point(km, orc):
    X = np.array([[1.5, -2.0, 3.0]], np.float32)
    diag = run_and_compare(km, orc, X, 1, 2.0, 2, 1)
    assert diag["final_cost"] == 0.0


def test_all_identical_points_warns(km, orc):
    X = np.full((300, 4), 2.5, np.float32)
    g = km.KMeansPar(_dev(X), 3, 6.0, 3, 1)
    for r in range(1, 4):
        assert g.round(r, sync=True) == (0, 0.0)
    assert g.weight() == 1
    C, st = g.recluster()
    assert st == km.KMPAR_WARN_FEW_CANDIDATES
    assert np.all(C.cpu().numpy() == 2.5)
    out = g.lloyd(C, 5)
    assert out["final_cost"] == 0.0
    g.close()


def test_huge_ell_takes_all_points(km, orc):
    # distinct grid points: every D^2 >= 1 > phi / l, so every p is capped at 1
    X = np.stack(np.meshgrid(np.arange(4), np.arange(5), np.arange(2)), -1).reshape(-1, 3).astype(np.float32)
    g = km.KMeansPar(_dev(X), 40, 3e4, 1, 3)
    na, phi = g.round(1, sync=True)
    assert na == 39 and phi == 0.0
    assert g.weight() == 40
    C, st = g.recluster()
    out = g.lloyd(C, 5)
    assert out["final_cost"] == 0.0
    g.close()


def test_state_machine_and_arguments(km):
    X = _dev(datagen.uniform_box(100, 2, seed=1))
    with pytest.raises(km.KmparError) as e:
        km.kmpar_init(X.data_ptr(), 0, 2, 3, 4.0, 2, 0, km.KMPAR_FP32)
    assert e.value.status == km.KMPAR_ERR_ARG
    with pytest.raises(km.KmparError) as e:
        km.kmpar_init(X.data_ptr(), 100, 2, 3, -1.0, 2, 0, km.KMPAR_FP32)
    assert e.value.status == km.KMPAR_ERR_ARG
    with pytest.raises(km.KmparError) as e:
        km.kmpar_init(X.data_ptr(), 100, 2, 3, 1e6, 2, 0, km.KMPAR_FP32)
    assert e.value.status == km.KMPAR_ERR_UNSUPPORTED
    g = km.KMeansPar(X, 3, 4.0, 2, 0)
    with pytest.raises(km.KmparError) as e:
        g.round(2)
    assert e.value.status == km.KMPAR_ERR_STATE
    with pytest.raises(km.KmparError) as e:
        g.weight()
    assert e.value.status == km.KMPAR_ERR_STATE
    g.round(1)
    with pytest.raises(km.KmparError) as e:
        g.recluster()
    assert e.value.status == km.KMPAR_ERR_STATE
    g.round(2)
    g.weight()
    with pytest.raises(km.KmparError) as e:
        g.round(3)
    assert e.value.status == km.KMPAR_ERR_STATE
    g.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_weighted_lloyd_on_candidates_matches_oracle(km, orc, precision):
    """Step 8's optional second half: Lloyd's iteration on the weighted candidates
    from the weighted k-means++ centers, against the oracle's from the same seed."""
    X = datagen.gauss_mixture(8000, 15, 30, 10.0, seed=61)
    Xd = _dev(X)
    g = km.KMeansPar(Xd, 30, 60.0, 5, 8, precision=precision)
    for r in range(1, 6):
        g.round(r)
    cand, w = g.candidates()
    C, _ = g.recluster()
    C0 = C.cpu().numpy().astype(np.float64)
    it = km.kmpar_weighted_lloyd(g.ctx, C.data_ptr(), 25)
    Cg = C.cpu().numpy()
    g.close()
    cand, w = cand.cpu().numpy(), w.cpu().numpy()
    oC, olab, oit, owc = orc.weighted_lloyd(X[cand], w, C0, 25)
    assert it == oit and it >= 1
    np.testing.assert_allclose(Cg, oC, rtol=1e-6, atol=1e-6 * (np.abs(oC).max() + 1))


def test_fit_with_weighted_lloyd_flag(km, orc):
    X = datagen.gauss_mixture(6000, 15, 25, 10.0, seed=62)
    n, d, k = X.shape[0], X.shape[1], 25
    Xd = _dev(X)
    Cd = torch.empty(k, d, dtype=torch.float32, device="cuda")
    r = km.kmpar_fit(Xd.data_ptr(), n, d, k, 50.0, 5, 3, km.KMPAR_FP32, 50, Cd.data_ptr(), None, flags=10 << 8)
    par = orc.kmeans_par(X, k, 50.0, 5, 3)
    oC, _, _, _ = orc.weighted_lloyd(X[par.cand], par.w, par.seed_centers.astype(np.float64), 10)
    _, _, oit, ofc, _, _ = orc.lloyd(X, oC, 50)
    assert math.isclose(r["final_cost"], ofc, rel_tol=1e-4)
