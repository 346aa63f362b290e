"""Pins of the oracle's lagged multi-guiding variant (a reordering of Sec.
2.1's generation: generation t >= 2 takes its guiding sparks from the
guiding vectors of generation t - 1 at the fireworks' current positions,
G_t = x_t + beta GV_{t-1}, so that explosion and guiding sparks can be
evaluated together; generation 1 runs the method as written).

The guiding vectors are pinned to a brute-force sort and FP32 sums in list
order, their composition with orc_guide_from to the pinned orc_guide, the
lagged guiding spark to x + GV in FP32 (beta = 1), and whole runs to the
method as written where the lag cannot matter (beta = 0, generation 1)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore")


def _case(seed, mu=3, lam=12, m=3, D=37, lb=-1.0, ub=1.0, beta=1.0, lagged=1, spread=0.6):
    p = oracle.make_params(dim=D, lb=lb, ub=ub, mu=mu, lam=lam, m=m, beta=beta, lagged_guiding=lagged)
    rng = np.random.default_rng(seed)
    fw_x = rng.uniform(lb, ub, size=(mu, D)).astype(np.float32)
    fw_a = np.full(mu, spread, np.float32)
    sparks = oracle.explode(p, seed, 1, fw_x, fw_a)
    fit = rng.standard_normal(mu * lam).astype(np.float32)
    fit[::7] = fit[0]  # ties: the index decides
    return p, fw_x, fw_a, sparks, fit


def _brute_vectors(p, sparks, fit):
    """GV from first principles: sort each group by (fitness, index), sum the k best and the k worst rows
    in that order in FP32, divide by k in FP32."""
    g = p.lam // p.m
    gv = np.zeros((p.mu * p.m, p.dim), np.float32)
    for i in range(p.mu):
        for q in range(p.m):
            idx = np.arange(q * g, (q + 1) * g)
            f = fit[i * p.lam + idx]
            order = idx[np.lexsort((idx, f))]          # ascending fitness, then index
            top, bottom = order[:p.k], order[::-1][:p.k]
            st = sparks[i * p.lam + top[0]].copy()
            sb = sparks[i * p.lam + bottom[0]].copy()
            for r in range(1, p.k):
                st = (st + sparks[i * p.lam + top[r]]).astype(np.float32)
                sb = (sb + sparks[i * p.lam + bottom[r]]).astype(np.float32)
            gv[i * p.m + q] = (st - sb) / np.float32(p.k)
    return gv


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_vectors_equal_brute_force(seed):
    p, _, _, sparks, fit = _case(seed, lam=20, m=2)  # g = 10, k = 2
    top, bottom = oracle.rank(p, fit)
    assert np.array_equal(oracle.guiding_vectors(p, sparks, top, bottom), _brute_vectors(p, sparks, fit))


@pytest.mark.parametrize("seed,beta,spread", [(4, 1.0, 0.6), (5, 1.7, 0.9), (6, 0.5, 0.05)])
def test_vectors_then_guide_from_is_the_guide(seed, beta, spread):
    """With the vectors of the same generation the two steps are the method's own guiding step, mapping
    draws included (wide amplitudes and beta > 1 push coordinates out of the box)."""
    p, fw_x, fw_a, sparks, fit = _case(seed, beta=beta, spread=spread)
    top, bottom = oracle.rank(p, fit)
    want = oracle.guide(p, seed, 5, fw_x, fw_a, sparks, top, bottom)
    got = oracle.guide_from(p, seed, 5, fw_x, fw_a, oracle.guiding_vectors(p, sparks, top, bottom))
    assert np.array_equal(want, got)


def test_lagged_generation_uses_the_previous_vectors():
    """Generation 2's guiding sparks are x_2 + GV_1 (beta = 1: one FP32 addition) wherever that stays in the
    box; elsewhere they are redrawn inside the firework's clipped amplitude box."""
    w = W.scaled(W.MLP_8_16_3, n_samples=64)
    prob = oracle.Problem.for_workload(w)
    p = oracle.params_for(w, lagged_guiding=1)
    seed = 11
    x, a = oracle.init(p, seed)
    f = prob.fitness_many(x).astype(np.float32)
    g1 = oracle.generation(p, prob, seed, 1, x, a, f)
    assert np.array_equal(g1["gv"], _brute_vectors(p, g1["sparks"], g1["fit_e"]))
    g2 = oracle.generation(p, prob, seed, 2, g1["fw_x"], g1["fw_amp"], g1["fw_f"], gv_prev=g1["gv"])
    xs = np.repeat(g1["fw_x"], p.m, axis=0)
    amp = np.repeat(g1["fw_amp"], p.m)[:, None]
    plain = (xs + g1["gv"]).astype(np.float32)
    inside = (plain >= p.lb) & (plain <= p.ub)
    assert inside.mean() > 0.5
    assert np.array_equal(g2["guides"][inside], plain[inside])
    lo = np.maximum(p.lb, xs - amp)
    hi = np.minimum(p.ub, xs + amp)
    out = ~inside
    assert np.all(g2["guides"][out] >= lo[out]) and np.all(g2["guides"][out] <= hi[out])
    # generation 2's own vectors come from its own sparks and ranks
    assert np.array_equal(g2["gv"], _brute_vectors(p, g2["sparks"], g2["fit_e"]))
    # and differ from what the method as written would have used
    p0 = oracle.params_for(w)
    g2_plain = oracle.generation(p0, prob, seed, 2, g1["fw_x"], g1["fw_amp"], g1["fw_f"])
    assert not np.array_equal(g2_plain["guides"], g2["guides"])
    assert np.array_equal(g2_plain["sparks"], g2["sparks"])


def test_generation_one_is_the_method():
    w = W.SPHERE_30
    prob = oracle.Problem.for_workload(w)
    seed = 3
    res = []
    for lag in (0, 1):
        p = oracle.params_for(w, lagged_guiding=lag)
        x, a = oracle.init(p, seed)
        f = prob.fitness_many(x).astype(np.float32)
        res.append(oracle.generation(p, prob, seed, 1, x, a, f))
    for key in ("sparks", "guides", "fw_x", "fw_amp", "fw_f", "winner"):
        assert np.array_equal(res[0][key], res[1][key]), key


def test_beta_zero_runs_agree():
    """With beta = 0 every guiding spark is its firework (inside the box, so never mapped), whatever the
    vectors: the lagged run is the method's run, generation for generation."""
    w = W.scaled(W.SPHERE_30, eval_budget=W.budget_for_generations(5, 40, 4, 25))
    prob = oracle.Problem.for_workload(w)
    r = [oracle.run(oracle.params_for(w, beta=0.0, lagged_guiding=lag), prob, 9, w.eval_budget, want_trace=True)
         for lag in (0, 1)]
    assert np.array_equal(r[0]["trace"], r[1]["trace"])
    assert np.array_equal(r[0]["best_x"], r[1]["best_x"]) and r[0]["evals"] == r[1]["evals"]


def test_lagged_run_budget_and_descent():
    """The variant spends the budget exactly as the method does and still converges on the sphere."""
    w = W.SPHERE_30
    prob = oracle.Problem.for_workload(w)
    r0 = oracle.run(oracle.params_for(w), prob, 0, w.eval_budget)
    r1 = oracle.run(oracle.params_for(w, lagged_guiding=1), prob, 0, w.eval_budget, want_trace=True)
    assert r1["evals"] == r0["evals"] and r1["gens"] == r0["gens"]
    assert np.all(np.diff(r1["trace"]) <= 0)
    assert r1["best_f"] < 1e-4
