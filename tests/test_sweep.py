"""The rounds/oversampling sweep (Sec. 5.3, Fig. 5.2).  On the CPU the oracle runs
the sweep's grid on GAUSSMIXTURE data and the figure's shape is checked: while
r l < k too few candidates exist and the cost is poor; once r l >= k it drops
sharply and then stays flat.  On the GPU the package's sweep (through kmpar_fit)
must give the same candidates and costs as the oracle on the same grid."""
import math
import statistics

import numpy as np
import pytest

from paper_1203_6402_gb300 import datagen

K = 20
ROUNDS = [1, 2, 3, 5, 8]
FACTORS = [0.25, 1.0]
SEEDS = list(range(11))   # 11 runs per point, as in Table 1


def _X():
    return datagen.gauss_mixture(3000, 15, K, 10.0, seed=2012)


def _oracle_sweep(orc, X):
    rows = {}
    for f in FACTORS:
        for r in ROUNDS:
            fin, cand = [], []
            for s in SEEDS:
                par, ll = orc.fit(X, K, f * K, r, s, 100)
                fin.append(ll["final_cost"])
                cand.append(len(par.cand))
            rows[(f, r)] = (statistics.median(fin), statistics.median(cand))
    return rows


@pytest.mark.slow
def test_sweep_shape_rounds_times_ell_against_k(orc):
    rows = _oracle_sweep(orc, _X())
    # l = k/4: r = 1 gives about 1 + l < k candidates, r = 8 about 1 + 8 l > k
    few, enough = rows[(0.25, 1)], rows[(0.25, 8)]
    assert few[1] < K <= enough[1]
    assert few[0] > 1.5 * enough[0], (few, enough)
    # once r l >= 2k the final cost is flat (within 30% across r and l; medians of
    # local optima), and every point with r l < k stays well above it
    good = [v[0] for (f, r), v in rows.items() if r * f >= 2]
    assert max(good) <= 1.3 * min(good), good
    bad = [v[0] for (f, r), v in rows.items() if r * f < 1]
    assert min(bad) > 1.4 * min(good), (bad, good)


@pytest.mark.gpu
def test_gpu_sweep_matches_oracle(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6402_gb300 import sweep
    X = _X()
    got = sweep.sweep(X, K, ROUNDS, FACTORS, SEEDS)
    ref = _oracle_sweep(orc, X)
    for w in got:
        fin, cand = ref[(w["ell_over_k"], w["r"])]
        assert w["candidates"] == cand
        assert math.isclose(w["final_cost"], fin, rel_tol=1e-4), (w, fin)
    assert "| l/k | r |" in sweep.table(got)
