"""Pins of the oracle's loser-out tournament (Algorithm 1, the step after the
selection; reading C-R15): a firework other than the run's best, with a
finite fitness before and after the selection, loses when its last
improvement I, extrapolated over the g_rem generations left, cannot reach
the run's best, fmaf(-I, g_rem, f) > best; a loser is re-initialised
uniformly in the box with amplitude A0 and fitness +infinity."""
import numpy as np
import pytest
from scipy import stats

import oracle

pytestmark = pytest.mark.filterwarnings("ignore")


def _p(mu=4, dim=10, **kw):
    return oracle.make_params(dim=dim, lb=-1.0, ub=1.0, mu=mu, lam=8, m=2, loser_out=1, **kw)


def _lo(p, f_old, fw_f, run_best, g_rem, gen=3, seed=7):
    x = np.zeros((p.mu, p.dim), np.float32)
    a = np.full(p.mu, 0.3, np.float32)
    return oracle.loser_out(p, seed, gen, g_rem, run_best, np.float32(f_old), x, a, np.float32(fw_f))


def test_closed_form_decisions():
    # best firework 3 (0.5); I = 0.1, 0, 0.5; g_rem = 2: projections 0.7, 2.0, 1.5 all above 0.5
    _, a, f, lo = _lo(_p(), [1.0, 2.0, 3.0, 0.5], [0.9, 2.0, 2.5, 0.5], 0.5, 2)
    assert lo.tolist() == [1, 1, 1, 0]
    assert np.all(np.isinf(f[:3])) and f[3] == np.float32(0.5)
    assert np.all(a[:3] == np.float32(2.0)) and a[3] == np.float32(0.3)
    # g_rem = 10: 0.9 - 1.0 = -0.1 and 2.5 - 5.0 = -2.5 reach the best, the stalled firework does not
    _, _, _, lo = _lo(_p(), [1.0, 2.0, 3.0, 0.5], [0.9, 2.0, 2.5, 0.5], 0.5, 10)
    assert lo.tolist() == [0, 1, 0, 0]


def test_projection_equal_to_best_is_kept():
    # I = 0.25 exactly, g_rem = 2: 1.0 - 0.5 = 0.5, not above the best 0.5
    _, _, _, lo = _lo(_p(mu=2), [1.25, 0.5], [1.0, 0.5], 0.5, 2)
    assert lo.tolist() == [0, 0]
    _, _, _, lo = _lo(_p(mu=2), [1.25, 0.5], [1.0, 0.5], 0.4999, 2)
    assert lo.tolist() == [1, 0]


def test_no_time_left_keeps_only_the_best_ones():
    # g_rem = 0: the projection is the fitness itself
    _, _, _, lo = _lo(_p(mu=4), [1.0, 0.7, 0.5, 0.9], [1.0, 0.7, 0.5, 0.5], 0.5, 0)
    assert lo.tolist() == [1, 1, 0, 0]   # firework 2 is the first minimum; 3 ties the best, proj not above


def test_best_firework_never_loses():
    # the run's best-so-far (0.1) is below every firework: only the first minimum (index 1) is spared
    _, _, _, lo = _lo(_p(mu=3), [2.0, 1.0, 1.0], [2.0, 1.0, 1.0], 0.1, 5)
    assert lo.tolist() == [1, 0, 1]


def test_non_finite_fitness_is_not_judged():
    f_old = [np.inf, 2.0, np.nan, 0.5]
    fw_f = [0.9, np.nan, 2.5, 0.5]
    _, _, _, lo = _lo(_p(), f_old, fw_f, 0.5, 1)
    assert lo.tolist() == [0, 0, 0, 0]


def test_reinitialised_positions_are_uniform_in_the_box():
    p = _p(mu=2, dim=40000)
    x, _, _, lo = _lo(p, [2.0, 0.5], [2.0, 0.5], 0.5, 3, gen=5)
    assert lo.tolist() == [1, 0]
    assert np.all(x[1] == 0.0)          # the best firework's row is untouched
    v = x[0].astype(np.float64)
    assert v.min() >= -1.0 and v.max() < 1.0
    assert stats.kstest((v + 1.0) / 2.0, "uniform").pvalue > 1e-3
    x2, _, _, _ = _lo(p, [2.0, 0.5], [2.0, 0.5], 0.5, 3, gen=6)
    assert not np.array_equal(x[0], x2[0])   # another generation draws another position
    x3, _, _, _ = _lo(p, [2.0, 0.5], [2.0, 0.5], 0.5, 3, gen=5)
    assert np.array_equal(x[0], x3[0])       # and the same one the same


def test_runs_keep_budget_and_never_lose_their_best():
    import workloads as W
    w = W.scaled(W.MLP_8_16_3, eval_budget=6000)
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    on = oracle.run(oracle.params_for(w, loser_out=1), prob, 3, w.eval_budget, want_trace=True)
    off = oracle.run(oracle.params_for(w), prob, 3, w.eval_budget, want_trace=True)
    assert on["evals"] == off["evals"] and on["gens"] == off["gens"]
    assert np.all(np.diff(on["trace"]) <= 0)
    assert abs(on["best_f"] - prob.fitness(on["best_x"])) < 1e-12
