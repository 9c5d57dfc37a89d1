"""Parity at full size: the whole path (Alg. 2 steps 1-8, then Lloyd) on the
KDD-shaped workloads of 1,000,000 x 42 (k = 500, the benchmark's configuration
and launch) and 4,800,000 x 42 (k = 1000), split-BF16 screening.  The oracle
cannot run these, so sampled outputs are checked one by one against a brute-force
FP64 scan, and properties that hold at any size are checked on every point:
phi = sum D^2 (Sec. 3.1), sum w = n and w = counts of idx (Alg. 2 step 7), seed
centers are candidate rows (step 8), Lloyd's cost never increases and equals the
exact cost of its labels.  At 1e6 points the FP32 CUDA-core path must take the
very same decisions."""
import math

import numpy as np
import pytest

from paper_1203_6402_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SAMPLE = 2000


@pytest.fixture(scope="module")
def km():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6402_gb300 import kmpar
    kmpar.load()
    return kmpar


def _nearest_fp64(Xs, C):
    """Brute force: per sampled row the best and second-best exact d^2 and the best
    center (lowest number on ties)."""
    Xs = Xs.astype(np.float64)
    C = C.astype(np.float64)
    bj, b1, b2 = [], [], []
    step = max(1, 4_000_000 // (C.shape[0] * C.shape[1]))   # rows per chunk: ~32 MB of differences
    for i in range(0, len(Xs), step):
        D = ((Xs[i:i + step, None, :] - C[None, :, :]) ** 2).sum(-1)
        order = np.argsort(D, axis=1, kind="stable")[:, :2]
        bj.append(order[:, 0])
        b1.append(np.take_along_axis(D, order[:, :1], 1)[:, 0])
        b2.append(np.take_along_axis(D, order[:, 1:2], 1)[:, 0] if C.shape[0] > 1 else np.full(len(D), np.inf))
    return np.concatenate(bj), np.concatenate(b1), np.concatenate(b2)


def _run(km, X, Xd, k, ell, rounds, seed, precision, max_iter):
    g = km.KMeansPar(Xd, k, ell, rounds, seed, precision=precision)
    phis = []
    for r in range(1, rounds + 1):
        na, phi = g.round(r, sync=True)
        D2, _ = g.state()
        phis.append((phi, float(D2.double().sum())))
    D2, idx = g.state()
    cand, w = g.candidates()
    C, st = g.recluster()
    out = g.lloyd(C.clone(), max_iter, labels=True, hist=True)
    res = dict(phis=phis, D2=D2, idx=idx, cand=cand, w=w, C=C, st=st, out=out, stats=g.stats())
    g.close()
    return res


def _check(X, Xd, res, k):
    n = X.shape[0]
    rng = np.random.default_rng(99)
    s = np.sort(rng.choice(n, SAMPLE, replace=False))
    # phi = sum D^2 after every round (the library sums FP32 D^2 in FP64 in a fixed tree)
    for phi, ref in res["phis"]:
        assert math.isclose(phi, ref, rel_tol=1e-9), (phi, ref)
    D2 = res["D2"].cpu().numpy()
    idx = res["idx"].cpu().numpy()
    cand = res["cand"].cpu().numpy()
    w = res["w"].cpu().numpy()
    assert np.isfinite(D2).all() and (D2 >= 0).all()
    # step 7: weights are the counts of the nearest-candidate numbers
    assert w.sum() == n
    assert np.array_equal(w, np.bincount(idx, minlength=len(cand)))
    # D^2 and idx of sampled points against a brute-force scan of every candidate
    bj, b1, b2 = _nearest_fp64(X[s], X[cand])
    tie = b2 <= b1 * (1 + 1e-6)
    assert np.all((idx[s] == bj) | tie), np.flatnonzero((idx[s] != bj) & ~tie)[:5]
    np.testing.assert_allclose(D2[s], b1, rtol=1e-5, atol=1e-30)
    # step 8: every seed center is a candidate row
    C = res["C"].cpu().numpy()
    rows = {X[j].tobytes() for j in cand}
    assert all(C[i].tobytes() in rows for i in range(k))
    # Lloyd: monotone cost, exact cost of the final labels, sampled labels nearest
    out = res["out"]
    hist = np.array(out["cost_hist"])
    assert np.all(np.diff(hist) <= 1e-6 * hist[0])
    return s, out["labels"], hist


@pytest.mark.parametrize("name,max_iter", [("kdd_n1M_d42_k500", 100), ("kdd_n4.8M_d42_k1000", 20)])
def test_full_size_properties_and_samples(km, name, max_iter):
    w = datagen.WORKLOADS[name]
    X = datagen.make(name, seed=1000)
    Xd = torch.from_numpy(X).cuda()
    g = km.KMeansPar(Xd, w["k"], w["ell"], w["rounds"], 7, precision="bf16x3")
    phis = []
    for r in range(1, w["rounds"] + 1):
        na, phi = g.round(r, sync=True)
        D2, _ = g.state()
        phis.append((phi, float(D2.double().sum())))
    D2, idx = g.state()
    cand, wt = g.candidates()
    C, st = g.recluster()
    C0 = C.clone()
    out = g.lloyd(C, max_iter, labels=True, hist=True)
    stats = g.stats()
    g.close()
    res = dict(phis=phis, D2=D2, idx=idx, cand=cand, w=wt, C=C0, st=st, out=out)
    s, lab, hist = _check(X, Xd, res, w["k"])
    # the final cost is the exact cost of the final labels against the final centers
    Cf = C.double()
    labt = lab.long()
    exact = float(((Xd.double() - Cf[labt]) ** 2).sum())
    assert math.isclose(out["final_cost"], exact, rel_tol=1e-5), (out["final_cost"], exact)
    # sampled labels are the nearest final centers (ties aside)
    bj, b1, b2 = _nearest_fp64(X[s], C.cpu().numpy())
    tie = b2 <= b1 * (1 + 1e-6)
    labs = lab.cpu().numpy()[s]
    assert np.all((labs == bj) | tie), np.flatnonzero((labs != bj) & ~tie)[:5]
    assert stats["screen_rows"] > 0


def test_full_size_tensor_path_takes_the_fp32_decisions(km):
    """1e6 x 42, k = 500: candidates, weights, seed centers, Lloyd labels and cost
    are identical whether the distances are screened on the tensor cores (split
    BF16 or plain BF16, exact refine) or computed in FP32 on CUDA cores."""
    name = "kdd_n1M_d42_k500"
    w = datagen.WORKLOADS[name]
    X = datagen.make(name, seed=1000)
    Xd = torch.from_numpy(X).cuda()
    res = {}
    for prec in ("fp32", "bf16x3", "bf16"):
        res[prec] = _run(km, X, Xd, w["k"], w["ell"], w["rounds"], 7, prec, 30)
    a = res["fp32"]
    for prec in ("bf16x3", "bf16"):
        b = res[prec]
        assert torch.equal(a["cand"], b["cand"]) and torch.equal(a["w"], b["w"]), prec
        assert torch.equal(a["idx"], b["idx"]) and torch.equal(a["D2"], b["D2"]), prec
        assert torch.equal(a["C"], b["C"]), prec
        assert torch.equal(a["out"]["labels"], b["out"]["labels"]), prec
        assert a["out"]["final_cost"] == b["out"]["final_cost"] and a["out"]["iters"] == b["out"]["iters"], prec


def test_large_k_wide_rows(km):
    """The shape of the 1e7 x 128, k = 1e4, l = 2e4 configuration at n = 2e6
    (plain BF16 screening): 79 streamed center tiles per Lloyd pass and ~21,000
    per round batch, per-row refine copies, ~1e5 candidates reclustered by the
    cooperative grid kernel.  Same sampled and whole-set checks."""
    n, d, k, ell = 2_000_000, 128, 10_000, 20_000.0
    X = datagen.gauss_mixture(n, d, k, 100.0, seed=1234)
    Xd = torch.from_numpy(X).cuda()
    g = km.KMeansPar(Xd, k, ell, 5, 11, precision="bf16")
    phis = []
    for r in range(1, 6):
        na, phi = g.round(r, sync=True)
        D2, _ = g.state()
        phis.append((phi, float(D2.double().sum())))
    D2, idx = g.state()
    cand, wt = g.candidates()
    C, st = g.recluster()
    C0 = C.clone()
    out = g.lloyd(C, 3, labels=True, hist=True)
    stats = g.stats()
    g.close()
    assert len(cand) > 50_000
    for phi, ref in phis:
        assert math.isclose(phi, ref, rel_tol=1e-9), (phi, ref)
    D2h, idxh, candh, wh = D2.cpu().numpy(), idx.cpu().numpy(), cand.cpu().numpy(), wt.cpu().numpy()
    assert np.isfinite(D2h).all() and (D2h >= 0).all()
    assert wh.sum() == n and np.array_equal(wh, np.bincount(idxh, minlength=len(candh)))
    rng = np.random.default_rng(5)
    s = np.sort(rng.choice(n, 200, replace=False))
    bj, b1, b2 = _nearest_fp64(X[s], X[candh])
    tie = b2 <= b1 * (1 + 1e-6)
    assert np.all((idxh[s] == bj) | tie)
    np.testing.assert_allclose(D2h[s], b1, rtol=1e-5, atol=1e-30)
    rows = {X[j].tobytes() for j in candh}
    C0h = C0.cpu().numpy()
    assert all(C0h[i].tobytes() in rows for i in range(k))
    hist = np.array(out["cost_hist"])
    assert np.all(np.diff(hist) <= 1e-6 * hist[0])
    labs = out["labels"]
    exact = float(((Xd.double() - C.double()[labs.long()]) ** 2).sum())
    assert math.isclose(out["final_cost"], exact, rel_tol=1e-5), (out["final_cost"], exact)
    bj, b1, b2 = _nearest_fp64(X[s], C.cpu().numpy())
    tie = b2 <= b1 * (1 + 1e-6)
    assert np.all((labs.cpu().numpy()[s] == bj) | tie)
    # plain BF16 (error ~2^-6 of ||x'|| ||c'||) leaves many rows of the rounds to the
    # exact fix-up: their candidates are data points, about two per true cluster,
    # so the two nearest are often near ties; every row is decided exactly all the same
    # rows: 5 round passes and 4 Lloyd assignments (updates 0..3), each row of an
    # assignment after the first either screened or settled by Lloyd's bounds
    assert stats["screen_rows"] + stats["lloyd_settled"] == (5 + 4) * n
    assert stats["lloyd_settled"] > 0 and 0 < stats["screen_fallback"] < stats["screen_rows"]


def test_full_size_exact_rounds(km):
    """Exactly-l rounds (Sec. 5.3) at 1e6 x 42, l = 1000: every round adds exactly
    1000 points never drawn before, phi = sum D^2, sum w = n; round 1 draws what
    the oracle draws from its own FP64 D^2 (no boundary near-tie); the split-BF16
    path takes the FP32 path's draws, D^2 and idx."""
    from oracle import oracle as orc
    name = "kdd_n1M_d42_k500"
    w = datagen.WORKLOADS[name]
    X = datagen.make(name, seed=1000)
    n, d = X.shape
    L = int(w["ell"])
    Xd = torch.from_numpy(X).cuda()
    res = {}
    for prec in ("fp32", "bf16x3"):
        g = km.KMeansPar(Xd, w["k"], w["ell"], w["rounds"], 7, precision=prec, sampling="exact")
        rounds = []
        for r in range(1, w["rounds"] + 1):
            na, phi = g.round(r, sync=True)
            D2, _ = g.state()
            rounds.append((na, phi, float(D2.double().sum())))
        cand, wt = g.candidates()
        D2, idx = g.state()
        res[prec] = (cand.cpu().numpy(), wt.cpu().numpy(), D2.cpu().numpy(), idx.cpu().numpy(), rounds)
        g.close()
    cand, wt, D2, idx, rounds = res["fp32"]
    assert [r[0] for r in rounds] == [L] * w["rounds"]
    for _, phi, ref in rounds:
        assert math.isclose(phi, ref, rel_tol=1e-9), (phi, ref)
    assert len(cand) == 1 + L * w["rounds"] and len(np.unique(cand)) == len(cand)
    assert wt.sum() == n and np.array_equal(wt, np.bincount(idx, minlength=len(cand)))
    for a, b in zip(res["fp32"][:4], res["bf16x3"][:4]):
        assert np.array_equal(a, b)
    # round 1 against the oracle: its own first center, FP64 D^2 and clocks
    i0 = orc.init_index(n, 7)
    assert cand[0] == i0
    D2o, _, _ = orc.init(X, i0)
    sel, near = orc.sample_exact(D2o, w["ell"], 1, 7, (2 * d + 16) * 2.0 ** -24)
    if not near:
        assert np.array_equal(cand[1:1 + L], sel)
