"""GPU parity of one MGFWA generation against the CPU oracle, through the C ABI.

Bar (per the method's arithmetic):
  * spark positions, guiding sparks, ranks, winners, amplitudes: bit-exact
    (both sides compute them with the same explicitly rounded FP32 steps);
  * rank and selection decisions: bit-exact once fed the oracle's fitness
    (rounded to FP32, the precision the kernels decide in);
  * FP32 fitness: within 1e-5 relative of the FP64 oracle plus an absolute
    floor of 1e-5 nats -- a K-term FP32 dot product carries about
    sqrt(K) 2^-24 relative error per hidden unit (~2e-6 at K = 784), and a
    sample's cross-entropy is a difference of logits of magnitude up to
    ~1e2, whose FP32 rounding (~1e2 x 2^-24 ~ 6e-6) bounds the absolute
    error once the loss itself is tiny (confidently classified samples);
  * FP64 reported best loss: within 1e-12 relative of the oracle.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

FP32_RTOL = 1e-5
FP32_ATOL = 1e-5


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2501_03944_gb300 as p
    return p


def _setup(w, seed):
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    p = oracle.params_for(w)
    return X, y, prob, p


def _rel(a, b, atol=FP32_ATOL):
    """|a - b| / (|b| + atol / rtol): <= FP32_RTOL means within rtol |b| + atol."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / (np.abs(b) + atol / FP32_RTOL)


SMALL_CASES = {
    "mlp8-16-3_N512": W.MLP_8_16_3,
    "mlp8-16-3_N300": W.scaled(W.MLP_8_16_3, n_samples=300),
    "mlp784-64-10_small": W.scaled(W.MLP_784_64_10, n_samples=200, n_fireworks=2, sparks_per_firework=24,
                                   guiding_per_firework=4),
    "mlp96-40-24-10_3layer": W.scaled(W.MLP_3072_128_64_10, widths=(96, 40, 24, 10), n_samples=129,
                                      n_fireworks=3, sparks_per_firework=16, guiding_per_firework=2),
    "gfwa_m1_g64": W.scaled(W.MLP_8_16_3, n_fireworks=2, sparks_per_firework=64, guiding_per_firework=1),
    "g2_k1_mu1_N1": W.scaled(W.MLP_8_16_3, n_samples=1, n_fireworks=1, sparks_per_firework=8,
                             guiding_per_firework=4),
    "odd_dim_8-3-2": W.scaled(W.MLP_8_16_3, widths=(8, 3, 2), n_samples=64),
    "sphere30": W.SPHERE_30,
    # more fireworks per run than the selection stages in shared memory (its serial part reads them from
    # global memory then)
    "sphere30_mu1030": W.scaled(W.SPHERE_30, n_fireworks=1030, sparks_per_firework=4, guiding_per_firework=2,
                                eval_budget=W.budget_for_generations(1030, 4, 2, 5)),
}


@pytest.mark.parametrize("name", list(SMALL_CASES))
def test_generation_phase_by_phase(pkg, name):
    w = SMALL_CASES[name]
    seed = 1000 + len(name)
    X, y, prob, p = _setup(w, seed)
    with pkg.Mgfwa.for_workload(w, seed, X=X, y=y) as run:
        fw_x, fw_a = oracle.init(p, seed)
        assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_X), fw_x)
        assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_AMP), fw_a)
        fw_f64 = prob.fitness_many(fw_x)
        assert np.all(_rel(run.read(pkg.MGFWA_BUF_FW_F), fw_f64) <= FP32_RTOL)
        fw_f = fw_f64.astype(np.float32)
        run.write(pkg.MGFWA_BUF_FW_F, fw_f)
        for gen in (1, 2, 3):
            ref = oracle.generation(p, prob, seed, gen, fw_x, fw_a, fw_f)
            run.phase(pkg.MGFWA_PHASE_EXPLODE)
            assert np.array_equal(run.read(pkg.MGFWA_BUF_SPARKS), ref["sparks"]), f"sparks gen {gen}"
            run.phase(pkg.MGFWA_PHASE_EVAL_E)
            assert np.all(_rel(run.read(pkg.MGFWA_BUF_FIT_E), ref["fit_e64"]) <= FP32_RTOL)
            run.write(pkg.MGFWA_BUF_FIT_E, ref["fit_e"])
            run.phase(pkg.MGFWA_PHASE_RANK)
            assert np.array_equal(run.read(pkg.MGFWA_BUF_TOP), ref["top"])
            assert np.array_equal(run.read(pkg.MGFWA_BUF_BOTTOM), ref["bottom"])
            run.phase(pkg.MGFWA_PHASE_GUIDE)
            assert np.array_equal(run.read(pkg.MGFWA_BUF_GUIDES), ref["guides"]), f"guides gen {gen}"
            run.phase(pkg.MGFWA_PHASE_EVAL_G)
            assert np.all(_rel(run.read(pkg.MGFWA_BUF_FIT_G), ref["fit_g64"]) <= FP32_RTOL)
            run.write(pkg.MGFWA_BUF_FIT_G, ref["fit_g"])
            run.phase(pkg.MGFWA_PHASE_SELECT)
            assert np.array_equal(run.read(pkg.MGFWA_BUF_WINNER), ref["winner"])
            assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_X), ref["fw_x"])
            assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_AMP), ref["fw_amp"])
            assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_F), ref["fw_f"])
            fw_x, fw_a, fw_f = ref["fw_x"], ref["fw_amp"], ref["fw_f"]
        assert run.info().evals == w.n_fireworks + 3 * w.sparks_per_generation


@pytest.mark.parametrize("w", [
    W.scaled(W.MLP_8_16_3, lb=-2.0, ub=3.0, n_fireworks=5),
    W.scaled(W.MLP_784_64_10, n_samples=64, n_fireworks=5, sparks_per_firework=8, guiding_per_firework=2),
    W.scaled(W.MLP_784_64_10, n_samples=64, n_fireworks=5, sparks_per_firework=8, guiding_per_firework=2,
             lb=-0.5, ub=1.5),
], ids=["8-16-3_bounds_-2_3", "784-64-10", "784-64-10_bounds_-0.5_1.5"])
def test_explosion_across_amplitude_regimes(pkg, w):
    """Explosion sparks bit-exact for amplitudes from 1% of the box to beyond it (the sampler's mapping is
    drawn only where a warp needs it, always, or as the whole-box draw), symmetric and asymmetric bounds, rows
    shorter than one thread's coordinates and rows much longer."""
    seed = 77
    X, y, prob, p = _setup(w, seed)
    with pkg.Mgfwa.for_workload(w, seed, X=X, y=y) as run:
        fw_x, _ = oracle.init(p, seed)
        width = np.float32(w.ub) - np.float32(w.lb)
        fw_a = (np.array([0.01, 0.3, 0.9, 1.0, 1.7], np.float32) * width).astype(np.float32)
        fw_f = prob.fitness_many(fw_x).astype(np.float32)
        run.write(pkg.MGFWA_BUF_FW_AMP, fw_a)
        run.write(pkg.MGFWA_BUF_FW_F, fw_f)
        ref = oracle.generation(p, prob, seed, 1, fw_x, fw_a, fw_f)
        run.phase(pkg.MGFWA_PHASE_EXPLODE)
        got = run.read(pkg.MGFWA_BUF_SPARKS)
    assert np.array_equal(got, ref["sparks"])
    inside = got[:, :w.dim]
    assert np.all(inside >= np.float32(w.lb)) and np.all(inside <= np.float32(w.ub))


def test_rank_and_select_with_ties_and_nan(pkg):
    w = W.scaled(W.MLP_8_16_3, n_samples=64, n_fireworks=3, sparks_per_firework=24, guiding_per_firework=3)
    seed = 77
    X, y, prob, p = _setup(w, seed)
    rng = np.random.default_rng(0)
    with pkg.Mgfwa.for_workload(w, seed, X=X, y=y) as run:
        fw_x = run.read(pkg.MGFWA_BUF_FW_X)
        fw_a = run.read(pkg.MGFWA_BUF_FW_AMP)
        fw_f = np.array([2.0, np.nan, 1.0], np.float32)
        run.write(pkg.MGFWA_BUF_FW_F, fw_f)
        run.phase(pkg.MGFWA_PHASE_EXPLODE)
        run.phase(pkg.MGFWA_PHASE_EVAL_E)
        fe = rng.integers(0, 3, size=72).astype(np.float32)
        fe[[3, 17, 40]] = np.nan
        run.write(pkg.MGFWA_BUF_FIT_E, fe)
        run.phase(pkg.MGFWA_PHASE_RANK)
        top, bot = oracle.rank(p, fe)
        assert np.array_equal(run.read(pkg.MGFWA_BUF_TOP), top)
        assert np.array_equal(run.read(pkg.MGFWA_BUF_BOTTOM), bot)
        run.phase(pkg.MGFWA_PHASE_GUIDE)
        sparks = run.read(pkg.MGFWA_BUF_SPARKS)
        guides = oracle.guide(p, seed, 1, fw_x, fw_a, sparks, top, bot)
        assert np.array_equal(run.read(pkg.MGFWA_BUF_GUIDES), guides)
        run.phase(pkg.MGFWA_PHASE_EVAL_G)
        fg = np.array([0.0, 5.0, np.nan, 0.0, 0.0, 1.0, 2.0, 2.0, 2.0], np.float32)
        run.write(pkg.MGFWA_BUF_FIT_G, fg)
        run.phase(pkg.MGFWA_PHASE_SELECT)
        nx, na, nf, win = oracle.select(p, fe, fg, sparks, guides, fw_x, fw_a, fw_f)
        assert np.array_equal(run.read(pkg.MGFWA_BUF_WINNER), win)
        assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_X), nx)
        assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_AMP), na)
        got_f = run.read(pkg.MGFWA_BUF_FW_F)
        assert np.array_equal(np.isnan(got_f), np.isnan(nf)) and np.array_equal(got_f[~np.isnan(nf)], nf[~np.isnan(nf)])


@pytest.mark.parametrize("widths,acts,N", [((8, 16, 3), (0,), 1), ((8, 16, 3), (0,), 127), ((8, 16, 3), (1,), 129),
                                           ((784, 64, 10), (1,), 300), ((64, 192, 7), (0,), 130),
                                           ((3072, 128, 64, 10), (1, 1), 256), ((24, 16, 8, 5), (0, 1), 200)])
def test_fp32_fitness_against_oracle(pkg, widths, acts, N):
    w = W.scaled(W.MLP_3072_128_64_10, widths=widths, acts=acts, n_samples=N, n_fireworks=2,
                 sparks_per_firework=8, guiding_per_firework=2)
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    xs = W.random_vectors(20, w.dim, -1.0, 1.0, seed=N)
    xs[0] = 0.0
    with pkg.Mgfwa.for_workload(w, 5, X=X, y=y) as run:
        got = run.evaluate(xs, pkg.MGFWA_FP32)
    want = prob.fitness_many(xs, n_threads=8)
    assert abs(want[0] - math.log(widths[-1])) < 1e-12
    assert np.all(_rel(got, want) <= FP32_RTOL), np.max(_rel(got, want))


def test_full_size_784_64_10_sampled(pkg):
    """The 784-64-10 workload at full size (D = 50,890, N = 2048, 5 x 200 sparks + 5 x 8 guiding)."""
    w = W.MLP_784_64_10
    seed = 3
    X, y, prob, p = _setup(w, seed)
    with pkg.Mgfwa.for_workload(w, seed, X=X, y=y) as run:
        fw_x, fw_a = oracle.init(p, seed)
        assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_X), fw_x)
        fw_f = run.read(pkg.MGFWA_BUF_FW_F)
        assert np.all(_rel(fw_f, prob.fitness_many(fw_x, 8)) <= FP32_RTOL)
        run.phase(pkg.MGFWA_PHASE_EXPLODE)
        sparks = run.read(pkg.MGFWA_BUF_SPARKS)
        ref_sparks = oracle.explode(p, seed, 1, fw_x, fw_a)
        assert np.array_equal(sparks, ref_sparks)
        run.phase(pkg.MGFWA_PHASE_EVAL_E)
        fe = run.read(pkg.MGFWA_BUF_FIT_E)
        pick = np.random.default_rng(1).choice(len(fe), 12, replace=False)
        assert np.all(_rel(fe[pick], prob.fitness_many(sparks[pick], 8)) <= FP32_RTOL)
        run.phase(pkg.MGFWA_PHASE_RANK)
        top, bot = oracle.rank(p, fe)
        assert np.array_equal(run.read(pkg.MGFWA_BUF_TOP), top)
        run.phase(pkg.MGFWA_PHASE_GUIDE)
        guides = oracle.guide(p, seed, 1, fw_x, fw_a, sparks, top, bot)
        assert np.array_equal(run.read(pkg.MGFWA_BUF_GUIDES), guides)
        run.phase(pkg.MGFWA_PHASE_EVAL_G)
        fg = run.read(pkg.MGFWA_BUF_FIT_G)
        assert np.all(_rel(fg[:6], prob.fitness_many(guides[:6], 8)) <= FP32_RTOL)
        run.phase(pkg.MGFWA_PHASE_SELECT)
        nx, na, nf, win = oracle.select(p, fe, fg, sparks, guides, fw_x, fw_a, fw_f)
        assert np.array_equal(run.read(pkg.MGFWA_BUF_WINNER), win)
        assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_X), nx)
        bx, bf, ev = run.best()
        assert ev == 5 + 1040
        assert abs(bf - prob.fitness(bx)) <= 1e-12 * abs(bf)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sphere_converges_on_gpu(pkg, seed):
    w = W.SPHERE_30
    with pkg.Mgfwa.for_workload(w, seed) as run:
        run.run()
        bx, bf, ev = run.best()
    assert ev <= 100_000 and bf < 1e-6
    assert abs(bf - float(np.sum(bx.astype(np.float64) ** 2))) <= 1e-15


def test_whole_runs_match_oracle_distribution(pkg):
    """20 seeds of the 8-16-3 workload, whole runs: GPU FP32 vs oracle final fitness."""
    from scipy import stats
    w = W.MLP_8_16_3
    X, y, prob, p = _setup(w, 0)
    gpu, orc = [], []
    for seed in range(20):
        with pkg.Mgfwa.for_workload(w, seed, X=X, y=y) as run:
            run.run()
            _, bf, ev = run.best()
        assert ev == 19_805
        gpu.append(bf)
        orc.append(oracle.run(p, prob, seed, w.eval_budget, n_threads=8)["best_f"])
    gpu, orc = np.array(gpu), np.array(orc)
    assert stats.mannwhitneyu(gpu, orc).pvalue > 0.01
    lg, lo = np.log(np.median(gpu)), np.log(np.median(orc))
    assert abs(lg - lo) <= abs(lo) * 0.05 + 0.5


def test_budget_and_step_semantics(pkg):
    w = W.scaled(W.MLP_8_16_3, eval_budget=5 + 3 * 220 + 100)
    X, y = W.make_data(w)
    with pkg.Mgfwa.for_workload(w, 0, X=X, y=y) as run:
        assert run.step(2) == pkg.MGFWA_OK
        assert run.step(5) == pkg.MGFWA_OK      # stops after one more generation
        assert run.info().generations == 3 and run.info().evals == 665
        assert run.step(1) == pkg.MGFWA_EBUDGET
        with pytest.raises(pkg.MgfwaError):
            run.phase(pkg.MGFWA_PHASE_RANK)     # out of order
        _, _, ev = run.best()
        assert ev == 665


def test_best_never_worsens_and_reports_fp64(pkg):
    w = W.MLP_8_16_3
    X, y, prob, p = _setup(w, 0)
    with pkg.Mgfwa.for_workload(w, 9, X=X, y=y) as run:
        last = math.inf
        for _ in range(10):
            run.step(5)
            bx, bf, _ = run.best()
            assert bf <= last * (1 + 1e-6)
            assert abs(bf - prob.fitness(bx)) <= 1e-12 * max(abs(bf), 1e-300)
            last = bf
