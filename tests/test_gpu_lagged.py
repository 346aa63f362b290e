"""Lagged multi-guiding on the GPU against the oracle: fed the oracle's
fitness, every generation's explosion sparks, guiding sparks (from the
previous generation's vectors from generation 2 on), recorded guiding
vectors, winners, fireworks, amplitudes and fitness match bit for bit.
Also: the variant spends the budget as the method does, and the handle
refuses what it does not support with it (checkpoints, groups)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2501_03944_gb300 as p
    return p


CASES = {
    "mlp8-16-3": (W.scaled(W.MLP_8_16_3, n_samples=300, eval_budget=W.budget_for_generations(5, 40, 4, 5)), {}),
    "mlp784-64-10_bf16": (W.scaled(W.MLP_784_64_10, n_samples=200, n_fireworks=3, sparks_per_firework=24,
                                   guiding_per_firework=4, eval_budget=W.budget_for_generations(3, 24, 4, 4)),
                          {"bf16": True}),
    "sphere30_beta1.5": (W.scaled(W.SPHERE_30, eval_budget=W.budget_for_generations(5, 40, 4, 5)), {"beta": 1.5}),
}


@pytest.mark.parametrize("name", list(CASES))
def test_lagged_phase_by_phase(pkg, name):
    w, opt = CASES[name]
    seed = 515 + len(name)
    X, y = (None, None) if w.kind == W.KIND_SPHERE else W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    beta = opt.get("beta", 1.0)
    p = oracle.params_for(w, lagged_guiding=1, beta=beta)
    prec = pkg.MGFWA_BF16 if opt.get("bf16") else pkg.MGFWA_FP32
    gens = (w.eval_budget - w.n_fireworks) // w.sparks_per_generation
    with pkg.Mgfwa.for_workload(w, seed, precision=prec, X=X, y=y, lagged_guiding=1, boost=beta,
                                elite_rescore=0) as run:
        fw_x, fw_a = oracle.init(p, seed)
        fw_f = prob.fitness_many(fw_x).astype(np.float32)
        run.write(pkg.MGFWA_BUF_FW_F, fw_f)
        gv = None
        for gen in range(1, gens + 1):
            ref = oracle.generation(p, prob, seed, gen, fw_x, fw_a, fw_f, gv_prev=gv)
            run.phase(pkg.MGFWA_PHASE_EXPLODE)
            assert np.array_equal(run.read(pkg.MGFWA_BUF_SPARKS), ref["sparks"]), gen
            if gen > 1:  # the lagged guiding sparks exist right after the explosion
                assert np.array_equal(run.read(pkg.MGFWA_BUF_GUIDES), ref["guides"]), gen
            run.phase(pkg.MGFWA_PHASE_EVAL_E)
            run.write(pkg.MGFWA_BUF_FIT_E, ref["fit_e"])
            run.phase(pkg.MGFWA_PHASE_RANK)
            assert np.array_equal(run.read(pkg.MGFWA_BUF_TOP).ravel(), ref["top"].ravel()), gen
            run.phase(pkg.MGFWA_PHASE_GUIDE)
            assert np.array_equal(run.read(pkg.MGFWA_BUF_GV), ref["gv"]), gen
            assert np.array_equal(run.read(pkg.MGFWA_BUF_GUIDES), ref["guides"]), gen
            run.phase(pkg.MGFWA_PHASE_EVAL_G)
            run.write(pkg.MGFWA_BUF_FIT_G, ref["fit_g"])
            run.phase(pkg.MGFWA_PHASE_SELECT)
            assert np.array_equal(run.read(pkg.MGFWA_BUF_WINNER), ref["winner"]), gen
            assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_X), ref["fw_x"]), gen
            assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_AMP), ref["fw_amp"]), gen
            assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_F), ref["fw_f"]), gen
            fw_x, fw_a, fw_f, gv = ref["fw_x"], ref["fw_amp"], ref["fw_f"], ref["gv"]
        assert run.info().evals == w.n_fireworks + gens * w.sparks_per_generation


def test_lagged_with_the_loser_out_tournament(pkg):
    """Both variants on: a re-drawn firework's next guiding sparks come from the recorded vectors at its
    new position (the mapping draws inside its reset amplitude box), bit for bit as in the oracle."""
    w = W.scaled(W.MLP_8_16_3, n_samples=300, eval_budget=W.budget_for_generations(5, 40, 4, 5))
    seed = 77
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    p = oracle.params_for(w, lagged_guiding=1, loser_out=1)
    g_max = oracle.g_max(p, w.eval_budget)
    losers = 0
    with pkg.Mgfwa.for_workload(w, seed, X=X, y=y, lagged_guiding=1, loser_out=1) as run:
        fw_x, fw_a = oracle.init(p, seed)
        fw_f = prob.fitness_many(fw_x).astype(np.float32)
        run.write(pkg.MGFWA_BUF_FW_F, fw_f)
        rb = fw_f[int(np.argmin([np.inf if np.isnan(f) else f for f in fw_f]))]
        run.write(pkg.MGFWA_BUF_BEST_F, np.array([rb], np.float32))
        gv = None
        for gen in range(1, g_max + 1):
            ref = oracle.generation(p, prob, seed, gen, fw_x, fw_a, fw_f, run_best=rb, g_rem=max(0, g_max - gen),
                                    gv_prev=gv)
            for ph, buf, key in ((pkg.MGFWA_PHASE_EXPLODE, None, None), (pkg.MGFWA_PHASE_EVAL_E, pkg.MGFWA_BUF_FIT_E,
                                                                      "fit_e"),
                                 (pkg.MGFWA_PHASE_RANK, None, None), (pkg.MGFWA_PHASE_GUIDE, None, None),
                                 (pkg.MGFWA_PHASE_EVAL_G, pkg.MGFWA_BUF_FIT_G, "fit_g")):
                run.phase(ph)
                if buf is not None:
                    run.write(buf, ref[key])
            assert np.array_equal(run.read(pkg.MGFWA_BUF_GUIDES), ref["guides"]), gen
            run.phase(pkg.MGFWA_PHASE_SELECT)
            assert np.array_equal(run.read(pkg.MGFWA_BUF_LOSER), ref["loser"]), gen
            assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_X), ref["fw_x"]), gen
            assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_AMP), ref["fw_amp"]), gen
            assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_F), ref["fw_f"]), gen
            losers += int(ref["loser"].sum())
            fw_x, fw_a, fw_f, rb, gv = ref["fw_x"], ref["fw_amp"], ref["fw_f"], ref["run_best"], ref["gv"]
    assert losers > 0, "the case should make some fireworks lose"


def test_lagged_fitness_of_both_spark_sets_in_one_launch(pkg):
    """From generation 2 on, the explosion and guiding sparks' fitness comes from one launch and still
    equals the oracle's objective on the GPU's own sparks (FP32)."""
    w = W.scaled(W.MLP_8_16_3, n_samples=300, eval_budget=W.budget_for_generations(5, 40, 4, 5))
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    with pkg.Mgfwa.for_workload(w, 9, X=X, y=y, lagged_guiding=1) as run:
        run.step(1)
        for ph in (pkg.MGFWA_PHASE_EXPLODE, pkg.MGFWA_PHASE_EVAL_E):
            run.phase(ph)
        fe = run.read(pkg.MGFWA_BUF_FIT_E).astype(np.float64)
        fg = run.read(pkg.MGFWA_BUF_FIT_G).astype(np.float64)
        ref_e = prob.fitness_many(run.read(pkg.MGFWA_BUF_SPARKS))
        ref_g = prob.fitness_many(run.read(pkg.MGFWA_BUF_GUIDES))
        assert np.all(np.abs(fe - ref_e) <= 1e-5 * (np.abs(ref_e) + 1e-3))
        assert np.all(np.abs(fg - ref_g) <= 1e-5 * (np.abs(ref_g) + 1e-3))


def test_lagged_budget_and_refusals(pkg):
    w = W.scaled(W.MLP_8_16_3, eval_budget=W.budget_for_generations(5, 40, 4, 12))
    X, y = W.make_data(w)
    with pkg.Mgfwa.for_workload(w, 4, X=X, y=y, lagged_guiding=1) as a, \
            pkg.Mgfwa.for_workload(w, 4, X=X, y=y) as b:
        a.run()
        b.run()
        _, fa, ea = a.best()
        _, fb, eb = b.best()
        assert ea == eb == w.eval_budget
        assert np.isfinite(fa) and fa < np.log(3)
        with pytest.raises(pkg.MgfwaError):
            a.checkpoint()
        with pytest.raises(pkg.MgfwaError):
            pkg.Group([a, b])
