"""The loser-out tournament (Algorithm 1, the step after the selection) on
the GPU against the oracle: fed the oracle's fitness, every generation's
winners, losers, fireworks, amplitudes, fitness and best-so-far match bit
for bit (the decisions and the re-drawn positions are exact FP32 / Philox
arithmetic on both sides).  The budgets are tight, so few generations are
left and fireworks lose.  Also: the tournament costs no evaluations, a
batch of runs ends where each run ends alone, and it can be switched off."""
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


def _key(f):
    return np.inf if np.isnan(f) else f


CASES = {
    "mlp8-16-3": W.scaled(W.MLP_8_16_3, n_samples=300, eval_budget=W.budget_for_generations(5, 40, 4, 4)),
    "mlp784-64-10": W.scaled(W.MLP_784_64_10, n_samples=200, n_fireworks=4, sparks_per_firework=24,
                             guiding_per_firework=4, eval_budget=W.budget_for_generations(4, 24, 4, 5)),
    "sphere30": W.scaled(W.SPHERE_30, eval_budget=W.budget_for_generations(5, 40, 4, 4)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_tournament_phase_by_phase(pkg, name):
    w = CASES[name]
    seed = 4242 + len(name)
    X, y = (None, None) if w.kind == W.KIND_SPHERE else W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    p = oracle.params_for(w, loser_out=1)
    g_max = oracle.g_max(p, w.eval_budget)
    losers = 0
    with pkg.Mgfwa.for_workload(w, seed, X=X, y=y, loser_out=1) as run:
        fw_x, fw_a = oracle.init(p, seed)
        fw_f = (prob.fitness_many(fw_x)).astype(np.float32)
        run.write(pkg.MGFWA_BUF_FW_F, fw_f)
        rb = fw_f[int(np.argmin([_key(f) for f in fw_f]))]
        run.write(pkg.MGFWA_BUF_BEST_F, np.array([rb], np.float32))
        for gen in range(1, g_max + 1):
            ref = oracle.generation(p, prob, seed, gen, fw_x, fw_a, fw_f, run_best=rb, g_rem=max(0, g_max - gen))
            for ph, buf, key in ((pkg.MGFWA_PHASE_EXPLODE, None, None), (pkg.MGFWA_PHASE_EVAL_E, pkg.MGFWA_BUF_FIT_E, "fit_e"),
                                 (pkg.MGFWA_PHASE_RANK, None, None), (pkg.MGFWA_PHASE_GUIDE, None, None),
                                 (pkg.MGFWA_PHASE_EVAL_G, pkg.MGFWA_BUF_FIT_G, "fit_g")):
                run.phase(ph)
                if buf is not None:
                    run.write(buf, ref[key])
            run.phase(pkg.MGFWA_PHASE_SELECT)
            assert np.array_equal(run.read(pkg.MGFWA_BUF_WINNER), ref["winner"]), gen
            assert np.array_equal(run.read(pkg.MGFWA_BUF_LOSER), ref["loser"]), gen
            assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_X), ref["fw_x"]), gen
            assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_AMP), ref["fw_amp"]), gen
            assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_F), ref["fw_f"]), gen
            assert run.read(pkg.MGFWA_BUF_BEST_F)[0] == ref["run_best"], gen
            losers += int(ref["loser"].sum())
            fw_x, fw_a, fw_f, rb = ref["fw_x"], ref["fw_amp"], ref["fw_f"], ref["run_best"]
        assert run.info().evals == w.n_fireworks + g_max * w.sparks_per_generation
    assert losers > 0, "the case should make some fireworks lose"


def test_tournament_costs_no_evaluations_and_keeps_the_best(pkg):
    w = W.scaled(W.MLP_8_16_3, eval_budget=6000)
    X, y = W.make_data(w)
    res = {}
    for lo in (0, 1):
        with pkg.Mgfwa.for_workload(w, 5, X=X, y=y, loser_out=lo) as h:
            h.run()
            x, f, ev = h.best()
            res[lo] = (h.info().generations, ev, f)
    assert res[0][:2] == res[1][:2]
    assert np.isfinite(res[1][2])


def test_tournament_batch_equals_runs_made_alone(pkg):
    w = W.scaled(W.MLP_8_16_3, n_samples=300, eval_budget=W.budget_for_generations(5, 40, 4, 6))
    X, y = W.make_data(w)
    B, seed = 3, 77
    with pkg.Mgfwa.for_workload(w, seed, X=X, y=y, n_runs=B, loser_out=1) as h:
        h.run()
        batched = [h.best(b) for b in range(B)]
        fw = h.read(pkg.MGFWA_BUF_FW_X).reshape(B, w.n_fireworks, -1)
    for b in range(B):
        with pkg.Mgfwa.for_workload(w, seed + b, X=X, y=y, loser_out=1) as h1:
            h1.run()
            x1, f1, e1 = h1.best()
            assert np.array_equal(h1.read(pkg.MGFWA_BUF_FW_X), fw[b])
        bx, bf, be = batched[b]
        assert np.array_equal(bx, x1) and bf == f1 and be == e1


def test_tournament_rejects_other_values(pkg):
    w = W.MLP_8_16_3
    X, y = W.make_data(w)
    with pytest.raises(pkg.MgfwaError):
        pkg.Mgfwa.for_workload(w, 1, X=X, y=y, loser_out=2)
