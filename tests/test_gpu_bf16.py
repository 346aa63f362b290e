"""GPU parity of the BF16 tensor-core fitness path (tcgen05 + TMA) against the
FP64 oracle, through the C ABI.

Bar: per-spark fitness within 1e-2 relative of the oracle (BF16 operands,
FP32 accumulation), plus an absolute floor of 1e-3 nats for samples whose
loss is tiny.  The 1e-2 bar is for batches of many samples, whose
independent rounding errors average out in the mean loss.  A batch of few
samples keeps the full per-sample error, so below 128 samples the bar is
6 sigma of a rounding model instead (`bf16_sigma`): every BF16 rounding
(unit roundoff u = 2^-8) is an independent error of variance (u v)^2 / 3 on
the value v it rounds -- both operands of layer 1, and on the two-layer
CTA-pair kernel also the activations and W2 of layer 2 -- propagated in FP64
through the weights, the ReLU and the softmax gradient of the loss.  Sampling, ranking, guiding and
selection are the same kernels as the FP32 path and stay bit-exact when fed
the oracle's fitness.  The tensor-core result is deterministic: the same
sparks give bitwise the same fitness on every call.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

BF16_RTOL = 1e-2
BF16_ATOL = 1e-3


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2501_03944_gb300 as p
    return p


def bf16_sigma(w, X, y, xs):
    """Standard deviation of each spark's BF16 loss error under the rounding model of the docstring
    (two-layer ReLU/tanh nets; FP64 throughout, from the inputs alone)."""
    d, h1, C = w.widths
    u2 = (2.0 ** -8) ** 2 / 3.0
    Xd = X.astype(np.float64)
    out = np.zeros(len(xs))
    for r, v in enumerate(np.asarray(xs, np.float64)):
        o = 0
        W1 = v[o:o + h1 * d].reshape(h1, d); o += h1 * d
        b1 = v[o:o + h1]; o += h1
        W2 = v[o:o + C * h1].reshape(C, h1); o += C * h1
        b2 = v[o:o + C]
        pre = Xd @ W1.T + b1
        if w.acts[0] == 1:
            h, slope = np.maximum(pre, 0.0), (pre > 0).astype(np.float64)
        else:
            h = np.tanh(pre)
            slope = 1.0 - h * h
        vh = slope ** 2 * ((Xd ** 2) @ (W1 ** 2).T) * 2 * u2            # layer 1: X and W1 rounded
        vz = vh @ (W2 ** 2).T + ((h ** 2) @ (W2 ** 2).T) * 2 * u2        # layer 2: activations and W2 rounded
        z = h @ W2.T + b2
        p = np.exp(z - z.max(1, keepdims=True))
        p /= p.sum(1, keepdims=True)
        p[np.arange(len(y)), y] -= 1.0                                   # d loss / d z per sample
        out[r] = np.sqrt(((p ** 2) * vz).sum(1).sum()) / len(y)
    return out


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / (np.abs(b) + BF16_ATOL / BF16_RTOL)


@pytest.mark.parametrize("widths,acts,N,count", [
    ((784, 64, 10), (1,), 200, 24),        # one sample tile (ragged), a few spark tiles
    ((784, 64, 10), (1,), 2048, 56),       # 16 sample tiles
    ((8, 32, 3), (0,), 300, 56),           # K = 8 < one K block (TMA zero fill), 5 sparks per tile, tanh
    ((64, 32, 7), (0,), 129, 24),          # ragged tail of one sample
    ((96, 128, 5), (1,), 1, 16),           # a single sample
    ((48, 128, 4), (1,), 260, 12),         # two sparks per tile, K = 48 inside one K block
    ((64, 64, 32, 5), (1, 0), 300, 24),    # three layers (ReLU, tanh): layers 2 and 3 on the tensor cores
    ((3072, 128, 64, 10), (1, 1), 256, 12),  # the 3072-128-64-10 network, one spark per tile
])
def test_bf16_fitness_against_oracle(pkg, widths, acts, N, count):
    w = W.scaled(W.MLP_784_64_10, widths=widths, acts=acts, n_samples=N, n_fireworks=2,
                 sparks_per_firework=count // 2 - 2, guiding_per_firework=2)
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    xs = W.random_vectors(count, w.dim, -1.0, 1.0, seed=N + count)
    xs[0] = 0.0
    with pkg.Mgfwa.for_workload(w, 5, precision=pkg.MGFWA_BF16, X=X, y=y) as run:
        got = run.evaluate(xs, pkg.MGFWA_BF16)
        again = run.evaluate(xs, pkg.MGFWA_BF16)
        f32 = run.evaluate(xs, pkg.MGFWA_FP32)
    want = prob.fitness_many(xs, n_threads=8)
    assert np.array_equal(got, again), "tensor-core fitness is not deterministic"
    assert abs(got[0] - np.log(widths[-1])) < 1e-6
    if N >= 128:
        err = _rel(got, want)
        assert np.all(err <= BF16_RTOL), (np.max(err), got[:4], want[:4])
    else:
        sig = bf16_sigma(w, X, y, xs)
        dev = np.abs(np.asarray(got, np.float64) - want)
        assert np.all(dev <= 6.0 * sig + BF16_ATOL), (np.max(dev / (sig + 1e-30)), got[:4], want[:4])
    assert np.all(np.abs(f32 - want) <= 1e-5 * np.abs(want) + 1e-5)


def test_bf16_rejects_unsupported_shapes(pkg):
    """The tensor-core path takes two-layer nets with h1 in {32, 64, 128} and three-layer nets with (h1, h2) in
    {(128, 64), (64, 32)} and at most 16 classes; others get EINVAL at create."""
    for widths, acts in (((8, 16, 3), (0,)), ((24, 16, 8, 5), (1, 1)), ((64, 48, 7), (1,)),
                         ((64, 64, 64, 5), (1, 1)), ((64, 64, 32, 20), (1, 1))):
        w = W.scaled(W.MLP_784_64_10, widths=widths, acts=acts, n_samples=64, n_fireworks=2,
                     sparks_per_firework=8, guiding_per_firework=2)
        X, y = W.make_data(w)
        with pytest.raises(pkg.MgfwaError) as e:
            pkg.Mgfwa.for_workload(w, 0, precision=pkg.MGFWA_BF16, X=X, y=y)
        assert e.value.status == pkg.MGFWA_EINVAL


def test_bf16_generation_phase_by_phase(pkg):
    w = W.scaled(W.MLP_784_64_10, n_samples=300, n_fireworks=3, sparks_per_firework=40, guiding_per_firework=4)
    seed = 21
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    p = oracle.params_for(w)
    with pkg.Mgfwa.for_workload(w, seed, precision=pkg.MGFWA_BF16, X=X, y=y) as run:
        fw_x, fw_a = oracle.init(p, seed)
        assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_X), fw_x)
        fw_f64 = prob.fitness_many(fw_x, 8)
        assert np.all(_rel(run.read(pkg.MGFWA_BUF_FW_F), fw_f64) <= BF16_RTOL)
        fw_f = fw_f64.astype(np.float32)
        run.write(pkg.MGFWA_BUF_FW_F, fw_f)
        for gen in (1, 2):
            ref = oracle.generation(p, prob, seed, gen, fw_x, fw_a, fw_f, n_threads=8)
            run.phase(pkg.MGFWA_PHASE_EXPLODE)
            assert np.array_equal(run.read(pkg.MGFWA_BUF_SPARKS), ref["sparks"])
            run.phase(pkg.MGFWA_PHASE_EVAL_E)
            assert np.all(_rel(run.read(pkg.MGFWA_BUF_FIT_E), ref["fit_e64"]) <= BF16_RTOL)
            run.write(pkg.MGFWA_BUF_FIT_E, ref["fit_e"])
            run.phase(pkg.MGFWA_PHASE_RANK)
            assert np.array_equal(run.read(pkg.MGFWA_BUF_TOP), ref["top"])
            run.phase(pkg.MGFWA_PHASE_GUIDE)
            assert np.array_equal(run.read(pkg.MGFWA_BUF_GUIDES), ref["guides"])
            run.phase(pkg.MGFWA_PHASE_EVAL_G)
            assert np.all(_rel(run.read(pkg.MGFWA_BUF_FIT_G), ref["fit_g64"]) <= BF16_RTOL)
            run.write(pkg.MGFWA_BUF_FIT_G, ref["fit_g"])
            run.phase(pkg.MGFWA_PHASE_SELECT)
            assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_X), ref["fw_x"])
            assert np.array_equal(run.read(pkg.MGFWA_BUF_FW_AMP), ref["fw_amp"])
            fw_x, fw_a, fw_f = ref["fw_x"], ref["fw_amp"], ref["fw_f"]


def test_bf16_full_size_784_64_10(pkg):
    """Full 784-64-10 workload (1000 explosion sparks x 2048 samples per launch): every explosion and guiding
    spark of the launch vs the oracle (about 6 s of FP64 on 16 host cores), and vs the FP32 path."""
    w = W.MLP_784_64_10
    seed = 4
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    with pkg.Mgfwa.for_workload(w, seed, precision=pkg.MGFWA_BF16, X=X, y=y) as run:
        run.phase(pkg.MGFWA_PHASE_EXPLODE)
        run.phase(pkg.MGFWA_PHASE_EVAL_E)
        sparks = run.read(pkg.MGFWA_BUF_SPARKS)
        fe = run.read(pkg.MGFWA_BUF_FIT_E)
        err = _rel(fe, prob.fitness_many(sparks[:len(fe)], 16))
        assert np.all(err <= BF16_RTOL), (int(np.argmax(err)), float(err.max()))
        for ph in (pkg.MGFWA_PHASE_RANK, pkg.MGFWA_PHASE_GUIDE, pkg.MGFWA_PHASE_EVAL_G, pkg.MGFWA_PHASE_SELECT):
            run.phase(ph)
        guides = run.read(pkg.MGFWA_BUF_GUIDES)
        fg = run.read(pkg.MGFWA_BUF_FIT_G)
        assert np.all(_rel(fg, prob.fitness_many(guides, 8)) <= BF16_RTOL)
        # BF16 and FP32 agree on every spark of the launch within the BF16 bar
        f32 = run.evaluate(sparks[:1000], pkg.MGFWA_FP32)
        assert np.all(_rel(fe, f32.astype(np.float64)) <= BF16_RTOL)


def test_bf16_full_size_3072_128_64_10(pkg):
    """The 3072-128-64-10 network at its full batch (N = 4096; 2 of its 8 fireworks, 512 explosion sparks per
    launch on the three-layer pair kernel): sampled sparks against the oracle, every spark against FP32."""
    w = W.scaled(W.MLP_3072_128_64_10, n_fireworks=2)
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    with pkg.Mgfwa.for_workload(w, 6, precision=pkg.MGFWA_BF16, X=X, y=y) as run:
        run.phase(pkg.MGFWA_PHASE_EXPLODE)
        run.phase(pkg.MGFWA_PHASE_EVAL_E)
        sparks = run.read(pkg.MGFWA_BUF_SPARKS)
        fe = run.read(pkg.MGFWA_BUF_FIT_E)
        n_e = len(fe)
        pick = np.concatenate([[0, 1], np.random.default_rng(3).choice(np.arange(2, n_e - 2), 6, replace=False),
                               [n_e - 2, n_e - 1]])
        assert np.all(_rel(fe[pick], prob.fitness_many(sparks[pick], 16)) <= BF16_RTOL)
        for ph in (pkg.MGFWA_PHASE_RANK, pkg.MGFWA_PHASE_GUIDE, pkg.MGFWA_PHASE_EVAL_G, pkg.MGFWA_PHASE_SELECT):
            run.phase(ph)
        f32 = run.evaluate(sparks[:n_e], pkg.MGFWA_FP32)
        assert np.all(_rel(fe, f32.astype(np.float64)) <= BF16_RTOL)


def test_bf16_whole_run_learns(pkg):
    w = W.scaled(W.MLP_784_64_10, eval_budget=W.budget_for_generations(5, 200, 8, 30))
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    with pkg.Mgfwa.for_workload(w, 11, precision=pkg.MGFWA_BF16, X=X, y=y) as run:
        f0 = float(np.min(run.read(pkg.MGFWA_BUF_FW_F)))
        run.run()
        bx, bf, ev = run.best()
    assert ev == w.eval_budget
    assert bf < 0.8 * f0
    assert abs(bf - prob.fitness(bx)) <= 1e-12 * bf


@pytest.mark.parametrize("N,mu,E,lam", [(300, 3, 3, 20), (2048, 5, 2, 20), (64, 2, 2, 2048)])
def test_elite_candidates_are_rescored_in_fp32(pkg, N, mu, E, lam):
    """With BF16 fitness, each firework's E best candidates (by BF16 fitness, (fitness, index) order) get their
    fitness recomputed by the FP32 path before selection; the others keep their BF16 values.  At 2048 samples
    the 10 re-scored rows x 16 sample tiles engage the FP32-accurate tensor-core first layer; at 300 samples
    the CUDA-core products run; with 2048 + 4 candidates a firework has more than the pick stages in shared
    memory."""
    import torch
    w = W.scaled(W.MLP_784_64_10, n_samples=N, n_fireworks=mu, sparks_per_firework=lam, guiding_per_firework=4)
    X, y = W.make_data(w)
    mu, lam, m = w.n_fireworks, w.sparks_per_firework, w.guiding_per_firework
    with pkg.Mgfwa.for_workload(w, 8, precision=pkg.MGFWA_BF16, X=X, y=y, elite_rescore=E) as run:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert run.fp32_tensor_cores() == (int(2 * mu * E * ((N + 127) // 128) >= sms), -1)
        for ph in (pkg.MGFWA_PHASE_EXPLODE, pkg.MGFWA_PHASE_EVAL_E, pkg.MGFWA_PHASE_RANK, pkg.MGFWA_PHASE_GUIDE,
                   pkg.MGFWA_PHASE_EVAL_G):
            run.phase(ph)
        fe, fg = run.read(pkg.MGFWA_BUF_FIT_E), run.read(pkg.MGFWA_BUF_FIT_G)
        sparks, guides = run.read(pkg.MGFWA_BUF_SPARKS), run.read(pkg.MGFWA_BUF_GUIDES)
        run.phase(pkg.MGFWA_PHASE_RESCORE)
        fe2, fg2 = run.read(pkg.MGFWA_BUF_FIT_E), run.read(pkg.MGFWA_BUF_FIT_G)
        run.phase(pkg.MGFWA_PHASE_SELECT)
        f32_e = run.evaluate(sparks, pkg.MGFWA_FP32)
        f32_g = run.evaluate(guides, pkg.MGFWA_FP32)
    for i in range(mu):
        cand = [(float(fe[i * lam + c]), c) for c in range(lam)] + [(float(fg[i * m + q]), lam + q) for q in range(m)]
        elite = {c for _, c in sorted(cand)[:E]}
        for c in range(lam + m):
            new = fe2[i * lam + c] if c < lam else fg2[i * m + c - lam]
            old = fe[i * lam + c] if c < lam else fg[i * m + c - lam]
            fp32 = f32_e[i * lam + c] if c < lam else f32_g[i * m + c - lam]
            if c in elite:
                # the re-score's FP32 sums run in another order than the FP32 kernel's: FP32 tolerance
                assert abs(new - fp32) <= 1e-5 * abs(fp32) + 1e-5, (i, c, new, fp32)
                assert new != old or abs(old - fp32) <= 1e-5 * abs(fp32) + 1e-5
            else:
                assert new == old, (i, c)
