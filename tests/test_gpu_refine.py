"""The learned part: hybrid refinement of each run's elite by projected
gradient descent (the gradient reading of the hybrid strategies of Sec. 5),
on the library's own FP32 backpropagation kernels.

* gradient parity: the kernels' FP32 objective and gradient against the
  oracle's FP64 backpropagation (itself pinned to torch autograd and central
  differences) on 2- and 3-layer nets, ragged batches and several vectors;
* the refinement phase against the oracle's refinement of the same elite;
* budget accounting of refining runs;
* the gain: at equal evaluation budget, MGFWA with refinement ends lower
  than MGFWA alone (20 seeds, a one-sided Mann-Whitney test)."""
import numpy as np
import pytest
from scipy import stats

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2501_03944_gb300 as p
    return p


def _net(widths, acts, N, lb=-1.0, ub=1.0, seed=0, **over):
    d = W.mlp_param_count(widths)
    kw = dict(name="t", kind=W.KIND_MLP_CE, widths=tuple(widths), acts=tuple(acts), n_samples=N, dim=d, lb=lb, ub=ub,
              n_fireworks=3, sparks_per_firework=8, guiding_per_firework=2, sigma=0.2, eval_budget=100_000,
              data_recipe="mixture", data_params=(2.0, 1.0), data_seed=seed)
    kw.update(over)
    return W.Workload(**kw)


def _sms():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("widths,acts,N,R", [
    ((8, 16, 3), (W.ACT_TANH,), 300, 3),
    ((16, 12, 8, 5), (W.ACT_TANH, W.ACT_RELU), 77, 2),
    ((64, 32, 7), (W.ACT_TANH,), 129, 4),
    ((784, 64, 10), (W.ACT_RELU,), 2048, 1),
    ((3072, 128, 64, 10), (W.ACT_RELU, W.ACT_RELU), 256, 1),
    ((8, 16, 3), (W.ACT_RELU,), 1, 1),
    # enough vectors x 128-sample tiles for the FP32-accurate tensor-core first layer:
    ((784, 64, 10), (W.ACT_RELU,), 1000, 10),                   # ragged tile (1000 = 7 x 128 + 104), ragged K
    ((64, 32, 7), (W.ACT_TANH,), 2000, 5),                      # h1 = 32, two K blocks
    ((40, 64, 5), (W.ACT_TANH,), 2048, 5),                      # second K block 8 wide
    ((32, 64, 5), (W.ACT_RELU,), 2048, 5),                      # one K block: no odd-block accumulator
    ((3072, 128, 64, 10), (W.ACT_TANH, W.ACT_TANH), 1024, 10),  # h1 = 128, 96 K blocks
    ((3072, 128, 64, 10), (W.ACT_RELU, W.ACT_RELU), 1024, 10),  # the same with ReLU: objective only (below)
])
def test_gradient_matches_oracle(pkg, widths, acts, N, R):
    """|dg| <= 1e-5 max|g| + 1e-4 |g|: every component is a sum over the N
    samples of products, accumulated in FP32 in tile and split order; with
    cancellation the sum of magnitudes can exceed the largest component by
    ~10^2, so ~sqrt(N) 2^-24 10^2 max|g| ~ 3e-7 max|g| is the expected size.
    The objective meets the FP32 fitness bar (1e-5 relative + 1e-5).  The
    first layer runs on the tensor cores (split TF32 products) exactly when
    its (128-sample tile, vector) pairs number half the SMs; the same bars
    hold on both paths.

    With ReLU, a pre-activation within its FP32 rounding of zero may take
    the other side of the kink than in FP64, which moves the gradient by one
    sample's whole contribution (~1/N of a typical component): any FP32
    evaluation does this at a rate of about one per 10^6 pre-activations.
    The 10 x 1024 x 128 first-layer pre-activations of the large ReLU case
    meet it, so there only the objective is compared; the same network with
    tanh checks the gradient through the same products."""
    w = _net(widths, acts, N)
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    xs = W.random_vectors(R, w.dim, -0.5, 0.5, 7)
    with pkg.Mgfwa.for_workload(w, 1, X=X, y=y, n_runs=R, refine_every=1, refine_steps=1, refine_lr=0.1) as h:
        f, g = h.gradient(xs)
        tc_expected = widths[1] in (32, 64, 128) and 2 * R * ((N + 127) // 128) >= _sms()
        assert h.fp32_tensor_cores() == (-1, int(tc_expected))
    for r in range(R):
        fo, go = oracle.gradient(prob, xs[r])
        assert abs(f[r] - fo) <= 1e-5 * abs(fo) + 1e-5
        if W.ACT_RELU in acts and R * N * widths[1] > 10 ** 6:
            continue
        mx = np.max(np.abs(go))
        assert np.all(np.abs(g[r] - go) <= 1e-5 * mx + 1e-4 * np.abs(go)), (r, np.max(np.abs(g[r] - go)) / mx)


@pytest.mark.parametrize("widths,acts,N,R", [
    ((784, 64, 10), (W.ACT_RELU,), 1000, 10),  # two vectors per tensor-core CTA
    ((64, 32, 7), (W.ACT_TANH,), 2000, 5),     # four per CTA, the last CTA with one
])
def test_tensor_core_layer_is_pairing_invariant(pkg, widths, acts, N, R):
    """The tensor-core first layer stacks 128 / h1 vectors in one CTA (N = 128 products); each vector's columns
    are its own sums, so a vector's objective and gradient are bitwise the same whichever vectors share its CTA."""
    w = _net(widths, acts, N)
    X, y = W.make_data(w)
    xs = W.random_vectors(R, w.dim, -0.5, 0.5, 11)
    perm = np.roll(np.arange(R), 3)
    with pkg.Mgfwa.for_workload(w, 1, X=X, y=y, n_runs=R, refine_every=1, refine_steps=1, refine_lr=0.1) as h:
        assert h.fp32_tensor_cores()[1] == int(2 * R * ((N + 127) // 128) >= _sms())
        f1, g1 = h.gradient(xs)
        f2, g2 = h.gradient(xs[perm])
    assert np.array_equal(f2, f1[perm]) and np.array_equal(g2, g1[perm])


def test_refine_phase_matches_oracle(pkg):
    w = W.scaled(W.MLP_8_16_3, n_fireworks=3, sparks_per_firework=12, guiding_per_firework=3)
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    p = oracle.params_for(w)
    B, seed, steps, lr = 2, 77, 5, 0.5
    mu = w.n_fireworks
    with pkg.Mgfwa.for_workload(w, seed, X=X, y=y, n_runs=B, refine_every=2, refine_steps=steps,
                                refine_lr=lr) as h:
        for gen in (1, 2):
            for ph in range(pkg.MGFWA_PHASE_SELECT + 1):
                h.phase(ph)
            if gen == 1:
                # not due: REFINE may be skipped, EXPLODE comes next
                continue
            fw_x = h.read(pkg.MGFWA_BUF_FW_X).reshape(B, mu, -1)
            fw_f = h.read(pkg.MGFWA_BUF_FW_F).reshape(B, mu)
            best_f = h.read(pkg.MGFWA_BUF_BEST_F)
            evals = h.info().evals
            h.phase(pkg.MGFWA_PHASE_REFINE)
            elite = h.read(pkg.MGFWA_BUF_REFINE_ELITE)
            rx = h.read(pkg.MGFWA_BUF_REFINE_X)
            rf = h.read(pkg.MGFWA_BUF_REFINE_F)
            nx = h.read(pkg.MGFWA_BUF_FW_X).reshape(B, mu, -1)
            nf = h.read(pkg.MGFWA_BUF_FW_F).reshape(B, mu)
            nbf = h.read(pkg.MGFWA_BUF_BEST_F)
            nbx = h.read(pkg.MGFWA_BUF_BEST_X)
            assert h.info().evals == evals + 3 * steps + 1
        for b in range(B):
            keys = np.where(np.isnan(fw_f[b]), np.inf, fw_f[b])
            e = int(np.argmin(keys))
            assert elite[b] == e
            ox, of = oracle.refine(prob, fw_x[b, e], steps, lr, w.lb, w.ub)
            # FP32 vs FP64 gradients (<= 1e-6 relative) over 5 steps of lr 0.5
            assert np.max(np.abs(rx[b] - ox)) <= 1e-5
            assert abs(rf[b] - of) <= 1e-5 * abs(of) + 1e-5
            take = rf[b] < fw_f[b, e]
            if take:
                assert np.array_equal(nx[b, e], rx[b]) and nf[b, e] == rf[b]
            else:
                assert np.array_equal(nx[b], fw_x[b]) and np.array_equal(nf[b], fw_f[b])
            others = [i for i in range(mu) if i != e]
            assert np.array_equal(nx[b, others], fw_x[b, others])
            if take and rf[b] < best_f[b]:
                assert nbf[b] == rf[b] and np.array_equal(nbx[b], rx[b])
            else:
                assert nbf[b] == best_f[b]


def test_refine_out_of_order_and_validation(pkg):
    w = W.MLP_8_16_3
    X, y = W.make_data(w)
    for over in (dict(refine_every=-1), dict(refine_every=2, refine_steps=0, refine_lr=0.1),
                 dict(refine_every=2, refine_steps=3, refine_lr=0.0)):
        with pytest.raises(pkg.MgfwaError):
            pkg.Mgfwa.for_workload(w, 0, X=X, y=y, **over)
    with pytest.raises(pkg.MgfwaError):
        pkg.Mgfwa.for_workload(W.SPHERE_30, 0, refine_every=1, refine_steps=1, refine_lr=0.1)
    with pkg.Mgfwa.for_workload(w, 0, X=X, y=y, refine_every=1, refine_steps=2, refine_lr=0.1) as h:
        for ph in range(pkg.MGFWA_PHASE_SELECT + 1):
            h.phase(ph)
        with pytest.raises(pkg.MgfwaError):
            h.phase(pkg.MGFWA_PHASE_EXPLODE)  # the due refinement may not be skipped
        h.phase(pkg.MGFWA_PHASE_REFINE)
        h.step(1)
    with pkg.Mgfwa.for_workload(w, 0, X=X, y=y) as h:
        with pytest.raises(pkg.MgfwaError):
            h.gradient(np.zeros((1, w.dim), np.float32))


@pytest.mark.parametrize("T,steps", [(1, 1), (3, 10), (4, 7)])
def test_budget_accounting_matches_oracle(pkg, T, steps):
    w = W.scaled(W.MLP_8_16_3, eval_budget=2500)
    X, y = W.make_data(w)
    pr = oracle.params_for(w, refine_every=T, refine_steps=steps, refine_lr=0.5)
    ref = oracle.run(pr, oracle.Problem.for_workload(w, X, y), 9, w.eval_budget)
    with pkg.Mgfwa.for_workload(w, 9, X=X, y=y, refine_every=T, refine_steps=steps, refine_lr=0.5) as h:
        h.run()
        info = h.info()
        _, _, evals = h.best()
    assert evals == ref["evals"] and info.generations == ref["gens"]


@pytest.mark.parametrize("case", ["mlp8-16-3 fp32, 3000 evaluations", "mlp784-64-10 bf16, 30 generations"])
def test_refinement_gains_at_equal_budget(pkg, case):
    if case.startswith("mlp8"):
        w, prec, T, steps, lr = W.scaled(W.MLP_8_16_3, eval_budget=3000), pkg.MGFWA_FP32, 3, 10, 0.5
    else:
        w, prec, T, steps, lr = (W.scaled(W.MLP_784_64_10, eval_budget=W.budget_for_generations(5, 200, 8, 30)),
                                 pkg.MGFWA_BF16, 5, 10, 0.05)
    X, y = W.make_data(w)
    plain, hybrid = [], []
    for seed in range(20):
        with pkg.Mgfwa.for_workload(w, 500 + seed, precision=prec, X=X, y=y) as h:
            h.run()
            plain.append(h.best()[1])
        with pkg.Mgfwa.for_workload(w, 500 + seed, precision=prec, X=X, y=y, refine_every=T, refine_steps=steps,
                                    refine_lr=lr) as h:
            h.run()
            _, f, ev = h.best()
            assert ev <= w.eval_budget
            hybrid.append(f)
    p = stats.mannwhitneyu(hybrid, plain, alternative="less").pvalue
    assert p < 0.01 and np.median(hybrid) < np.median(plain), (np.median(hybrid), np.median(plain), p)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_refining_batch_equals_runs_made_alone(pkg, precision):
    """Run b of a refining batch is bitwise the refining run seeded seed + b:
    the products' split-K chunks depend on their shapes only."""
    prec = {"fp32": pkg.MGFWA_FP32, "bf16": pkg.MGFWA_BF16}[precision]
    w = W.scaled(W.MLP_784_64_10, n_samples=300, n_fireworks=3, sparks_per_firework=20, guiding_per_firework=4,
                 eval_budget=W.budget_for_generations(3, 20, 4, 6) + 3 * 16)
    X, y = W.make_data(w)
    kw = dict(refine_every=2, refine_steps=5, refine_lr=0.05)
    B, seed = 3, 31
    with pkg.Mgfwa.for_workload(w, seed, precision=prec, X=X, y=y, n_runs=B, **kw) as h:
        h.run()
        batched = [h.best(b) for b in range(B)]
    for b in range(B):
        with pkg.Mgfwa.for_workload(w, seed + b, precision=prec, X=X, y=y, **kw) as h1:
            h1.run()
            x1, f1, e1 = h1.best()
        bx, bf, be = batched[b]
        assert np.array_equal(bx, x1) and bf == f1 and be == e1, b
