"""GPU parity of the FP8 (E4M3) tensor-core fitness path.

The FP8 path evaluates, exactly up to FP32 accumulation order and the TF32
second layer, the network whose X and first-layer weights are rounded to
E4M3 after scaling (X by 448 / max|X|, weights by 448 / max(|lb|, |ub|)),
with the first layer's sums scaled back before the bias.  The oracle's
fitness_fp8 computes that network in FP64 from its own pinned E4M3
quantizer, so the bar against it is the BF16 path's (1e-2 relative + 1e-3,
which covers the TF32 second layer).  Against the unquantized objective the
E4M3 rounding itself (2^-4 relative per value) moves the loss by up to
tens of percent; that bound is checked loosely.  Sampling, ranking, guiding
and selection are the kernels of the other paths; the elite re-score runs
in FP32 as on the BF16 path."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-2, 1e-3


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2501_03944_gb300 as p
    return p


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b) / (np.abs(b) + ATOL / RTOL)


@pytest.mark.parametrize("widths,acts,N,count", [
    ((784, 64, 10), (1,), 200, 24),        # one sample tile (ragged), several spark tiles; K tail of 16
    ((784, 64, 10), (1,), 2048, 56),       # 16 sample tiles
    ((16, 32, 3), (0,), 300, 56),          # K = 16 < one 128-element K block (TMA zero fill), tanh
    ((64, 32, 7), (0,), 129, 24),          # ragged tail of one sample
    ((48, 128, 4), (1,), 260, 12),         # two sparks per tile
    ((64, 64, 32, 5), (1, 0), 300, 24),    # three layers (ReLU, tanh)
    ((3072, 128, 64, 10), (1, 1), 256, 12),  # the 3072-128-64-10 network
])
def test_fp8_fitness_equals_quantized_oracle(pkg, widths, acts, N, count):
    w = W.scaled(W.MLP_784_64_10, widths=widths, acts=acts, n_samples=N, n_fireworks=2,
                 sparks_per_firework=count // 2 - 2, guiding_per_firework=2)
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    xs = W.random_vectors(count, w.dim, -1.0, 1.0, seed=N + count)
    xs[0] = 0.0
    with pkg.Mgfwa.for_workload(w, 5, precision=pkg.MGFWA_FP8, X=X, y=y) as run:
        info = run.info()
        got = run.evaluate(xs, pkg.MGFWA_FP8)
        again = run.evaluate(xs, pkg.MGFWA_FP8)
    assert info.fp8_inv_scale_w == np.float32(448.0) and info.fp8_inv_scale_x == np.float32(448.0 / np.abs(X).max())
    assert np.array_equal(got, again)
    want = np.array([oracle.fitness_fp8(prob, x, info.fp8_inv_scale_x, info.fp8_inv_scale_w) for x in xs])
    assert np.all(_rel(got, want) <= RTOL), np.max(_rel(got, want))
    exact = prob.fitness_many(xs, n_threads=8)
    assert np.all(np.abs(got - exact) <= 0.3 * np.abs(exact) + 0.05)


def test_fp8_full_size_3072_128_64_10(pkg):
    """The 3072-128-64-10 network at its full batch (N = 4096, 2 of 8 fireworks): sampled explosion sparks
    against the oracle's quantized network."""
    w = W.scaled(W.MLP_3072_128_64_10, n_fireworks=2)
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    with pkg.Mgfwa.for_workload(w, 7, precision=pkg.MGFWA_FP8, X=X, y=y, elite_rescore=0) as run:
        info = run.info()
        run.phase(pkg.MGFWA_PHASE_EXPLODE)
        run.phase(pkg.MGFWA_PHASE_EVAL_E)
        sparks = run.read(pkg.MGFWA_BUF_SPARKS)
        fe = run.read(pkg.MGFWA_BUF_FIT_E)
    pick = np.random.default_rng(4).choice(len(fe), 4, replace=False)
    want = np.array([oracle.fitness_fp8(prob, sparks[i], info.fp8_inv_scale_x, info.fp8_inv_scale_w) for i in pick])
    assert np.all(_rel(fe[pick], want) <= RTOL), np.max(_rel(fe[pick], want))


def test_fp8_full_size_784_64_10(pkg):
    """The bench's E4M3 launch: 784-64-10 at its full size (1000 explosion sparks x 2048 samples, 40 guiding
    sparks): the first and last sparks of the launch, 56 others and every guiding spark against the oracle's
    quantized network (the FP64 evaluations on host threads)."""
    from concurrent.futures import ThreadPoolExecutor
    w = W.MLP_784_64_10
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    with pkg.Mgfwa.for_workload(w, 9, precision=pkg.MGFWA_FP8, X=X, y=y, elite_rescore=0) as run:
        info = run.info()
        run.phase(pkg.MGFWA_PHASE_EXPLODE)
        run.phase(pkg.MGFWA_PHASE_EVAL_E)
        sparks = run.read(pkg.MGFWA_BUF_SPARKS)
        fe = run.read(pkg.MGFWA_BUF_FIT_E)
        for ph in (pkg.MGFWA_PHASE_RANK, pkg.MGFWA_PHASE_GUIDE, pkg.MGFWA_PHASE_EVAL_G):
            run.phase(ph)
        guides = run.read(pkg.MGFWA_BUF_GUIDES)
        fg = run.read(pkg.MGFWA_BUF_FIT_G)
    n = len(fe)
    pick = np.concatenate([np.arange(4), np.random.default_rng(8).choice(np.arange(4, n - 4), 56, replace=False),
                           np.arange(n - 4, n)])
    rows = [sparks[i] for i in pick] + list(guides[:len(fg)])
    with ThreadPoolExecutor(8) as ex:
        want = np.array(list(ex.map(
            lambda x: oracle.fitness_fp8(prob, x, info.fp8_inv_scale_x, info.fp8_inv_scale_w), rows)))
    got = np.concatenate([fe[pick], fg])
    err = _rel(got, want)
    assert np.all(err <= RTOL), (int(np.argmax(err)), float(err.max()))


def test_fp8_rejects_unaligned_inputs_and_other_precisions(pkg):
    w = W.scaled(W.MLP_784_64_10, widths=(8, 32, 3), acts=(0,), n_samples=64)
    X, y = W.make_data(w)
    with pytest.raises(pkg.MgfwaError) as e:
        pkg.Mgfwa.for_workload(w, 1, precision=pkg.MGFWA_FP8, X=X, y=y)
    assert e.value.status == pkg.MGFWA_EINVAL
    w2 = W.scaled(W.MLP_784_64_10, n_samples=64)
    X2, y2 = W.make_data(w2)
    with pkg.Mgfwa.for_workload(w2, 1, precision=pkg.MGFWA_FP8, X=X2, y=y2) as run:
        with pytest.raises(pkg.MgfwaError):
            run.evaluate(np.zeros((1, w2.dim), np.float32), pkg.MGFWA_BF16)
        run.evaluate(np.zeros((1, w2.dim), np.float32), pkg.MGFWA_FP32)


def test_fp8_generation_phase_by_phase(pkg):
    """Positions are the other paths' (bit-exact against the oracle when fed
    the oracle's fitness); the E best candidates are re-scored in FP32."""
    w = W.scaled(W.MLP_784_64_10, n_samples=300, n_fireworks=3, sparks_per_firework=20, guiding_per_firework=4)
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    p = oracle.params_for(w)
    seed = 14
    with pkg.Mgfwa.for_workload(w, seed, precision=pkg.MGFWA_FP8, X=X, y=y, elite_rescore=2) as run:
        fw_x, fw_a = oracle.init(p, seed)
        assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_X), fw_x)
        fw_f = prob.fitness_many(fw_x).astype(np.float32)
        run.write(pkg.MGFWA_BUF_FW_F, fw_f)
        ref = oracle.generation(p, prob, seed, 1, fw_x, fw_a, fw_f)
        run.phase(pkg.MGFWA_PHASE_EXPLODE)
        assert np.array_equal(run.read(pkg.MGFWA_BUF_SPARKS), ref["sparks"])
        run.phase(pkg.MGFWA_PHASE_EVAL_E)
        run.write(pkg.MGFWA_BUF_FIT_E, ref["fit_e"])
        run.phase(pkg.MGFWA_PHASE_RANK)
        run.phase(pkg.MGFWA_PHASE_GUIDE)
        assert np.array_equal(run.read(pkg.MGFWA_BUF_GUIDES), ref["guides"])
        run.phase(pkg.MGFWA_PHASE_EVAL_G)
        run.write(pkg.MGFWA_BUF_FIT_G, ref["fit_g"])
        run.phase(pkg.MGFWA_PHASE_SELECT)  # the re-score is skipped: selection on the injected fitness
        assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_X), ref["fw_x"])
        assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_AMP), ref["fw_amp"])


def test_fp8_whole_run_learns_and_batches(pkg):
    w = W.scaled(W.MLP_784_64_10, n_samples=300, n_fireworks=3, sparks_per_firework=20, guiding_per_firework=4,
                 eval_budget=W.budget_for_generations(3, 20, 4, 12))
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    with pkg.Mgfwa.for_workload(w, 3, precision=pkg.MGFWA_FP8, X=X, y=y, n_runs=2) as run:
        f0 = run.read(pkg.MGFWA_BUF_FW_F).min()
        run.run()
        batched = [run.best(b) for b in range(2)]
    for b in range(2):
        with pkg.Mgfwa.for_workload(w, 3 + b, precision=pkg.MGFWA_FP8, X=X, y=y) as r1:
            r1.run()
            x1, f1, e1 = r1.best()
        assert np.array_equal(batched[b][0], x1) and batched[b][1] == f1
        assert f1 < f0
        assert abs(f1 - prob.fitness(x1)) <= 1e-12 * abs(f1)  # the reported loss is the FP64 one
