"""Whole runs in the low precisions against the FP32 path: 20 seeds of the
784-64(ReLU)-10 workload (N = 2048, 5 fireworks x (200 + 8) sparks), 30
generations each, final best fitness (the FP64 report of the returned
vector).  BF16 and E4M3 fitness, each with the FP32 re-score of every
firework's elite candidates before selection, against the FP32 path:
Mann-Whitney U p > 0.01 and log-medians within 5% (+0.05).  The runs of one
seed diverge across precisions (their fitness values differ, so their
selections do), so the comparison is between distributions."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

SEEDS = range(20)
GENS = 30


@pytest.fixture(scope="module")
def finals():
    import __graft_entry__ as g
    g.build()
    import paper_2501_03944_gb300 as pkg
    w = W.scaled(W.MLP_784_64_10, eval_budget=W.budget_for_generations(5, 200, 8, GENS))
    X, y = W.make_data(w)
    out = {}
    for name, prec in (("fp32", pkg.MGFWA_FP32), ("bf16", pkg.MGFWA_BF16), ("fp8", pkg.MGFWA_FP8)):
        vals = []
        for seed in SEEDS:
            with pkg.Mgfwa.for_workload(w, 4000 + seed, precision=prec, X=X, y=y) as run:
                run.run()
                _, bf, _ = run.best()
                assert run.info().generations == GENS
            vals.append(bf)
        out[name] = np.array(vals)
    return out


@pytest.mark.parametrize("low", ["bf16", "fp8"])
def test_low_precision_runs_match_the_fp32_path(finals, low):
    from scipy import stats
    a, b = finals[low], finals["fp32"]
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(b))
    assert stats.mannwhitneyu(a, b).pvalue > 0.01, (np.median(a), np.median(b))
    la, lb = np.log(np.median(a)), np.log(np.median(b))
    assert abs(la - lb) <= abs(lb) * 0.05 + 0.05, (np.median(a), np.median(b))
