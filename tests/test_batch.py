"""kmpar_batch_run: many independent k-means|| problems in one call (Alg. 2 and
Lloyd per problem).  A seeded subset of the batched configuration (uneven n, d in
{32, 64, 128}, k log-uniform in [16, 256], l = 2k, r = 5, 10 Lloyd updates) is run
through the C ABI and every problem is compared with the FP64 oracle run on its
own rows: candidate sets and weights bit-exact, the seed cost within 1e-6 and the
final cost within 1e-4 relative (trajectories may part only at reported near
ties), final labels the nearest of the final centers."""
import math

import numpy as np
import pytest

from paper_1203_6402_gb300 import datagen

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def km():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6402_gb300 import kmpar
    kmpar.load()
    return kmpar


def _layout(km, probs):
    off = 0
    for p in probs:
        p["cand_offset"] = off
        off += km.kmpar_batch_cand_capacity(p["ell"], p["rounds"])
    return off


@pytest.mark.gpu
def test_batch_matches_oracle_per_problem(km, orc):
    probs = datagen.batched_problems(64, seed=3, n_lo=1_000, n_hi=6_000)
    X = datagen.batched_points(probs)
    ncand = _layout(km, probs)
    Xd = torch.from_numpy(X).cuda()
    C = torch.zeros(sum(p["k"] * p["d"] for p in probs), dtype=torch.float32, device="cuda")
    L = torch.zeros(sum(p["n"] for p in probs), dtype=torch.int32, device="cuda")
    cand = torch.full((ncand,), -1, dtype=torch.int32, device="cuda")
    w = torch.zeros(ncand, dtype=torch.int64, device="cuda")
    st, res = km.kmpar_batch_run(Xd.data_ptr(), probs, C.data_ptr(), L.data_ptr(), cand.data_ptr(), w.data_ptr())
    assert st in (km.KMPAR_OK, km.KMPAR_WARN_FEW_CANDIDATES)
    C, L, cand, w = C.cpu().numpy(), L.cpu().numpy(), cand.cpu().numpy(), w.cpu().numpy()
    parted = 0
    for p, r in zip(probs, res):
        n, d, k = p["n"], p["d"], p["k"]
        Xi = X[p["x_offset"]: p["x_offset"] + n * d].reshape(n, d)
        par = orc.kmeans_par(Xi, k, p["ell"], p["rounds"], p["seed"])
        m = r["m"]
        gc = cand[p["cand_offset"]: p["cand_offset"] + m]
        gw = w[p["cand_offset"]: p["cand_offset"] + m]
        if r["sample_near"] == 0:
            assert m == len(par.cand) and np.array_equal(gc, par.cand), p
            assert np.array_equal(gw, par.w)
        assert gw.sum() == n
        Cf = C[p["c_offset"]: p["c_offset"] + k * d].reshape(k, d)
        lab = L[p["l_offset"]: p["l_offset"] + n]
        chosen, rnear, _ = orc.recluster(Xi[par.cand].astype(np.float64), par.w, k, p["seed"])
        seed = Xi[par.cand[chosen]].astype(np.float64)
        oC, olab, oit, ofc, ohist, onear = orc.lloyd(Xi, seed, p["max_iter"])
        if r["recluster_near"] == 0 and not rnear.any():
            assert math.isclose(r["seed_cost"], orc.cost(Xi, seed), rel_tol=1e-6), p
            same = (r["iters"] == oit and math.isclose(r["final_cost"], ofc, rel_tol=1e-4))
            if same:
                np.testing.assert_allclose(Cf, oC, rtol=1e-5, atol=1e-5 * (np.abs(oC).max() + 1))
            else:
                # Lloyd's trajectories may part only at a near tie that either side reports
                # (the oracle keeps FP64 centers, the library rounds them to FP32)
                assert onear.any() or r["argmin_fp64"] > 0, (p, r, oit, ofc)
                assert r["final_cost"] <= r["seed_cost"] * (1 + 1e-6)
                parted += 1
        else:
            parted += 1
        # the final labels are the nearest of the final centers (FP64 check)
        D = ((Xi.astype(np.float64)[:, None, :] - Cf.astype(np.float64)[None]) ** 2).sum(-1)
        best = D.min(1)
        assert np.all(D[np.arange(n), lab] <= best * (1 + 1e-6) + 1e-30)
        assert math.isclose(r["final_cost"], best.sum(), rel_tol=1e-5)
    # most problems follow the oracle's trajectory to the end
    assert parted <= len(probs) // 4, parted


@pytest.mark.gpu
def test_batch_equals_single_problem_path(km):
    """Each problem's draws, candidates and weights equal those of kmpar_fit's FP32
    path run on that problem alone (the same counters and tie rules)."""
    probs = datagen.batched_problems(6, seed=9, n_lo=2_000, n_hi=20_000)
    X = datagen.batched_points(probs)
    ncand = _layout(km, probs)
    Xd = torch.from_numpy(X).cuda()
    C = torch.zeros(sum(p["k"] * p["d"] for p in probs), dtype=torch.float32, device="cuda")
    cand = torch.full((ncand,), -1, dtype=torch.int32, device="cuda")
    w = torch.zeros(ncand, dtype=torch.int64, device="cuda")
    st, res = km.kmpar_batch_run(Xd.data_ptr(), probs, C.data_ptr(), None, cand.data_ptr(), w.data_ptr())
    for p, r in zip(probs, res):
        n, d, k = p["n"], p["d"], p["k"]
        Xi = Xd[p["x_offset"]: p["x_offset"] + n * d].view(n, d)
        g = km.KMeansPar(Xi, k, p["ell"], p["rounds"], p["seed"], precision="fp32")
        for i in range(1, p["rounds"] + 1):
            g.round(i)
        gc, gw = g.candidates()
        Cs, _ = g.recluster()
        g.close()
        m = r["m"]
        assert m == len(gc)
        assert np.array_equal(cand[p["cand_offset"]: p["cand_offset"] + m].cpu().numpy(), gc.cpu().numpy())
        assert np.array_equal(w[p["cand_offset"]: p["cand_offset"] + m].cpu().numpy(), gw.cpu().numpy())


@pytest.mark.gpu
def test_batch_capacity_overflow_is_per_problem(km, monkeypatch):
    probs = datagen.batched_problems(3, seed=4, n_lo=3_000, n_hi=5_000, k_lo=20, k_hi=30)
    # a per-round capacity of 40 draws: problems 0 and 2 draw about 2 per round,
    # problem 1 about 200, so only its first round overflows
    monkeypatch.setenv("KMPAR_ROUND_CAPACITY", "40")
    probs[0]["ell"] = probs[2]["ell"] = 2.0
    probs[1]["ell"] = 200.0
    X = datagen.batched_points(probs)
    _layout(km, probs)
    Xd = torch.from_numpy(X).cuda()
    C = torch.zeros(sum(p["k"] * p["d"] for p in probs), dtype=torch.float32, device="cuda")
    st, res = km.kmpar_batch_run(Xd.data_ptr(), probs, C.data_ptr())
    assert st == km.KMPAR_ERR_CAPACITY
    assert res[1]["status"] == km.KMPAR_ERR_CAPACITY
    # about 11 candidates for k >= 20: these two finish with the few-candidates warning
    assert res[0]["status"] in (km.KMPAR_OK, km.KMPAR_WARN_FEW_CANDIDATES)
    assert res[2]["status"] in (km.KMPAR_OK, km.KMPAR_WARN_FEW_CANDIDATES)
    assert res[0]["final_cost"] > 0 and res[2]["final_cost"] > 0


def test_batched_problem_recipe():
    probs = datagen.batched_problems(4096, seed=1)
    n = np.array([p["n"] for p in probs])
    k = np.array([p["k"] for p in probs])
    d = np.array([p["d"] for p in probs])
    assert n.min() >= 1000 and n.max() <= 200_000 and set(d) == {32, 64, 128}
    assert k.min() >= 16 and k.max() <= 256 and all(p["ell"] == 2 * p["k"] for p in probs)
    # log-uniform n: the median sits near the geometric mean of the range
    assert 10_000 < np.median(n) < 18_000
    offs = [p["x_offset"] for p in probs]
    assert offs[0] == 0 and all(offs[i + 1] == offs[i] + n[i] * d[i] for i in range(len(probs) - 1))


def test_problem_struct_layout():
    import ctypes
    from paper_1203_6402_gb300 import kmpar
    assert ctypes.sizeof(kmpar.kmpar_problem) == 72
    assert kmpar.kmpar_problem.seed.offset == 40
    assert ctypes.sizeof(kmpar.kmpar_problem_result) == 56


@pytest.mark.gpu
def test_batch_clusters_equal_single_problem_path(km):
    """Problems of more than 25,000 rows run split over a thread-block cluster of 2,
    4 or 8 blocks (rows cut into contiguous ranges, draws appended rank by rank):
    draws, candidates and weights equal those of the
    single-problem FP32 path; Lloyd's labels and final cost agree closely."""
    probs = [dict(n=n, d=d, k=k, ell=2.0 * k, rounds=5, max_iter=10, seed=77 + i, data_seed=500 + i)
             for i, (n, d, k) in enumerate([(30_000, 32, 40), (70_000, 64, 90), (150_000, 128, 200),
                                            (200_000, 32, 16), (24_000, 128, 60)])]
    xo = co = lo = 0
    for p in probs:
        p.update(x_offset=xo, c_offset=co, l_offset=lo)
        xo += p["n"] * p["d"]
        co += p["k"] * p["d"]
        lo += p["n"]
    ncand = _layout(km, probs)
    X = datagen.batched_points(probs)
    Xd = torch.from_numpy(X).cuda()
    C = torch.zeros(co, dtype=torch.float32, device="cuda")
    L = torch.zeros(lo, dtype=torch.int32, device="cuda")
    cand = torch.full((ncand,), -1, dtype=torch.int32, device="cuda")
    w = torch.zeros(ncand, dtype=torch.int64, device="cuda")
    st, res = km.kmpar_batch_run(Xd.data_ptr(), probs, C.data_ptr(), L.data_ptr(), cand.data_ptr(), w.data_ptr())
    assert st in (km.KMPAR_OK, km.KMPAR_WARN_FEW_CANDIDATES)
    for p, r in zip(probs, res):
        n, d, k = p["n"], p["d"], p["k"]
        Xi = Xd[p["x_offset"]: p["x_offset"] + n * d].view(n, d)
        g = km.KMeansPar(Xi, k, p["ell"], p["rounds"], p["seed"], precision="fp32")
        for i in range(1, p["rounds"] + 1):
            g.round(i)
        gc, gw = g.candidates()
        Cs, _ = g.recluster()
        out = g.lloyd(Cs, p["max_iter"], labels=True)
        g.close()
        m = r["m"]
        assert m == len(gc), p
        assert np.array_equal(cand[p["cand_offset"]: p["cand_offset"] + m].cpu().numpy(), gc.cpu().numpy()), p
        assert np.array_equal(w[p["cand_offset"]: p["cand_offset"] + m].cpu().numpy(), gw.cpu().numpy()), p
        # Lloyd: the two paths round the centroids of equal sums differently in the last
        # bit (one compensated chain against 256-member pieces), so a near tie may part
        # them; the labels and costs must still agree closely
        assert abs(r["iters"] - out["iters"]) <= 1, (p, r)
        same = (L[p["l_offset"]: p["l_offset"] + n].cpu().numpy() == out["labels"].cpu().numpy()).mean()
        assert same >= 0.9999, (p, same)
        assert math.isclose(r["final_cost"], out["final_cost"], rel_tol=1e-6), (r, out["final_cost"])


def test_batch_tuning_table_and_split_setting():
    """The committed autotuner table names one of the measured thresholds, the one
    with the smallest time; the setter rejects a negative threshold."""
    from paper_1203_6402_gb300 import batch_tune
    t = batch_tune.load_table()
    assert t is not None and str(t["rows_per_block"]) in t["ms"]
    assert t["ms"][str(t["rows_per_block"])] == min(t["ms"].values())
    assert all(int(r) in batch_tune.CANDIDATES for r in t["ms"])
    from paper_1203_6402_gb300 import kmpar
    try:
        kmpar.load()
    except (FileNotFoundError, OSError):
        pytest.skip("library not built")
    with pytest.raises(kmpar.KmparError):
        kmpar.kmpar_batch_set_split(-1)
    kmpar.kmpar_batch_set_split(25000)
