"""Pins of the oracle's gradient and hybrid refinement (the learned part:
projected gradient descent on each run's elite, the gradient reading of the
hybrid strategies the paper's Sec. 5 proposes) against facts outside the
oracle: central differences of the oracle's own FP64 objective (itself
pinned to torch's float64 cross_entropy), torch float64 autograd (a library
routine), closed forms, and the clipping and descent properties of the
projected step."""
import numpy as np
import pytest

import workloads as W


def _net(widths, acts, n, seed, lo=-1.0, hi=1.0):
    d = W.mlp_param_count(widths)
    w = W.Workload(name="t", kind=W.KIND_MLP_CE, widths=tuple(widths), acts=tuple(acts), n_samples=n, dim=d,
                   lb=-5.0, ub=5.0, n_fireworks=1, sparks_per_firework=4, guiding_per_firework=1, sigma=0.2,
                   eval_budget=100, data_recipe="mixture", data_params=(2.0, 1.0), data_seed=seed)
    X, y = W.make_data(w)
    x = W.random_vectors(1, d, lo, hi, seed + 1)[0]
    return w, X, y, x


def _torch_grad(widths, acts, X, y, x):
    import torch
    import torch.nn.functional as F
    p = torch.tensor(x.astype(np.float64), requires_grad=True)
    a = torch.tensor(X.astype(np.float64))
    off = 0
    L = len(widths) - 1
    for l in range(L):
        fi, fo = widths[l], widths[l + 1]
        Wl = p[off:off + fi * fo].view(fo, fi)
        off += fi * fo
        bl = p[off:off + fo]
        off += fo
        a = F.linear(a, Wl, bl)
        if l + 1 < L:
            a = torch.tanh(a) if acts[l] == W.ACT_TANH else torch.relu(a)
    loss = F.cross_entropy(a, torch.tensor(y.astype(np.int64)))
    loss.backward()
    return loss.item(), p.grad.numpy()


@pytest.mark.parametrize("widths,acts", [((8, 16, 3), (W.ACT_TANH,)), ((8, 16, 3), (W.ACT_RELU,)),
                                         ((16, 12, 8, 5), (W.ACT_TANH, W.ACT_RELU)),
                                         ((8, 6, 7, 4), (W.ACT_RELU, W.ACT_TANH))])
def test_gradient_equals_torch_autograd(orc, widths, acts):
    w, X, y, x = _net(widths, acts, 37, 11)
    prob = orc.Problem.for_workload(w, X, y)
    f, g = orc.gradient(prob, x)
    tf, tg = _torch_grad(widths, acts, X, y, x)
    assert abs(f - tf) <= 1e-12 * abs(tf)
    assert np.max(np.abs(g - tg)) <= 1e-12 * max(1.0, np.max(np.abs(tg)))


@pytest.mark.parametrize("widths,acts", [((8, 5, 3), (W.ACT_TANH,)), ((8, 4, 3, 3), (W.ACT_TANH, W.ACT_TANH))])
def test_gradient_equals_central_differences(orc, widths, acts):
    """Every coordinate: (f(x + h e_k) - f(x - h e_k)) / (actual FP32 step), h = 2^-9."""
    w, X, y, x = _net(widths, acts, 23, 5)
    prob = orc.Problem.for_workload(w, X, y)
    _, g = orc.gradient(prob, x)
    h = np.float32(2.0 ** -9)
    for k in range(w.dim):
        xp, xm = x.copy(), x.copy()
        xp[k] = x[k] + h
        xm[k] = x[k] - h
        cd = (prob.fitness(xp) - prob.fitness(xm)) / (float(xp[k]) - float(xm[k]))
        # truncation error ~ h^2 |f'''| / 6 ~ 1e-6 at these scales
        assert abs(cd - g[k]) <= 2e-5 * (1.0 + abs(g[k])), k


def test_gradient_closed_form_when_only_the_output_bias_is_set(orc):
    """Zero weights and hidden biases: every logit vector is b_L, so the output
    bias gradient is softmax(b_L) - class frequencies and every other
    component is exactly zero (act(0) = 0 for tanh and ReLU)."""
    widths = (8, 16, 3)
    w, X, y, _ = _net(widths, (W.ACT_TANH,), 50, 3)
    x = np.zeros(w.dim, np.float32)
    bL = np.array([0.5, -1.25, 2.0], np.float32)
    x[-3:] = bL
    prob = orc.Problem.for_workload(w, X, y)
    f, g = orc.gradient(prob, x)
    sm = np.exp(bL.astype(np.float64) - bL.max())
    sm /= sm.sum()
    freq = np.bincount(y, minlength=3) / len(y)
    assert np.allclose(g[-3:], sm - freq, rtol=0, atol=1e-15)
    assert np.all(g[:-3] == 0.0)
    assert abs(f - float(np.mean(np.log(np.exp(bL.astype(np.float64)).sum()) - bL[y]))) < 1e-13
    # softmax minus one-hot sums to zero per sample
    assert abs(g[-3:].sum()) < 1e-15


def test_sphere_gradient(orc):
    prob = orc.Problem(orc.SPHERE, 30)
    x = W.random_vectors(1, 30, -5, 5, 9)[0]
    f, g = orc.gradient(prob, x)
    assert np.array_equal(g, 2.0 * x.astype(np.float64)) and f == prob.fitness(x)


def _fma32(a, b, c):
    """fmaf emulated in FP64: the FP32 product a*b is exact there; adding c and
    rounding twice (to FP64, then FP32) can differ from one rounding by one
    FP32 ulp, which the test's tolerance covers."""
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def test_refine_is_projected_gradient_descent(orc):
    """The oracle's refinement equals a plain loop over torch's gradient:
    w <- clip(fmaf(-lr, float32(g), w), lb, ub), two steps."""
    widths, acts = (8, 6, 3), (W.ACT_TANH,)
    w, X, y, x = _net(widths, acts, 29, 17, -2.0, 2.0)
    prob = orc.Problem.for_workload(w, X, y)
    lr, lb, ub = np.float32(0.75), np.float32(-2.0), np.float32(2.0)
    out, f = orc.refine(prob, x, 2, float(lr), float(lb), float(ub))
    ref = x.copy()
    for _ in range(2):
        _, tg = _torch_grad(widths, acts, X, y, ref)
        g32 = tg.astype(np.float32)
        ref = np.array([min(max(_fma32(-lr, g32[k], ref[k]), lb), ub) for k in range(w.dim)], np.float32)
    # torch's FP64 gradient may round to a neighbouring FP32 value: one ulp of lr*g
    assert np.max(np.abs(out - ref)) <= 1e-6
    assert abs(f - prob.fitness(out)) == 0.0


def test_refine_descends_and_stays_in_the_box(orc):
    w, X, y, x = _net((8, 16, 3), (W.ACT_TANH,), 64, 21)
    prob = orc.Problem.for_workload(w, X, y)
    same, f0 = orc.refine(prob, x, 0, 0.1, -5.0, 5.0)
    assert np.array_equal(same, x) and f0 == prob.fitness(x)
    prev = f0
    cur = x
    for _ in range(5):
        cur, f = orc.refine(prob, cur, 1, 0.05, -5.0, 5.0)
        assert f < prev
        prev = f
    big, _ = orc.refine(prob, x, 3, 1e4, -0.5, 0.5)
    assert big.min() >= -0.5 and big.max() <= 0.5
    assert np.mean(np.abs(big) == np.float32(0.5)) > 0.5  # most coordinates hit the box


def test_runs_with_refinement_charge_their_evaluations_and_gain(orc):
    w = W.scaled(W.MLP_8_16_3, eval_budget=3000)
    X, y = W.make_data(w)
    prob = orc.Problem.for_workload(w, X, y)
    T, Tg = 3, 10
    pr = orc.params_for(w, refine_every=T, refine_steps=Tg, refine_lr=0.5)
    p0 = orc.params_for(w)
    cost = orc.refine_cost(pr)
    assert cost == 3 * Tg + 1
    per = w.sparks_per_generation
    for seed in (1, 2):
        a = orc.run(pr, prob, seed, w.eval_budget)
        b = orc.run(p0, prob, seed, w.eval_budget)
        gens = a["gens"]
        assert a["evals"] == w.n_fireworks + gens * per + (gens // T) * cost <= w.eval_budget
        nxt = per + (cost if (gens + 1) % T == 0 else 0)
        assert a["evals"] + nxt > w.eval_budget
        assert a["best_f"] < b["best_f"]
