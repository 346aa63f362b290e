"""The paper's testbed objective (Sec. 4.1, Eq. 1: the scalar output of a
fixed network, minimised over its input) on the GPU against the oracle.

The GPU computes each layer in FP32: the fan-in split into four contiguous
chunks of 16 ceil(fan_in / 64), each a chain of fmaf in index order, the
chunk sums added in chunk order, then the bias and the activation; the
oracle in FP64.  The tolerance comes
from that arithmetic: every rounding is modelled as an independent error of
at most half an FP32 ulp of the value it rounds (variance |v|^2 2^-48 / 3),
propagated through the network's own weights and activation slopes in
FP64, and the test allows 10 of the resulting standard deviations (plus the
few-ulp error of FP32 tanh/erf at each activation).  A dropped term, a wrong
index or a wrong activation moves the output by far more."""
import math

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


_U = 2.0 ** -24  # FP32 unit roundoff


def _act(a, z):
    if a == W.ACT_RELU:
        return np.maximum(z, 0.0), (z > 0).astype(np.float64)
    if a == W.ACT_TANH:
        t = np.tanh(z)
        return t, 1.0 - t * t
    erf = np.vectorize(math.erf)(z / math.sqrt(2.0))
    pdf = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return 0.5 * z * (1.0 + erf), 0.5 * (1.0 + erf) + z * pdf


def fp32_sigma(w, params, x):
    """FP64 forward of one input with the standard deviation of the FP32
    forward's accumulated rounding error (the model in the module docstring)."""
    a = x.astype(np.float64)
    var = np.zeros_like(a)
    off = 0
    L = len(w.widths) - 1
    for l in range(L):
        fi, fo = w.widths[l], w.widths[l + 1]
        Wl = params[off:off + fi * fo].astype(np.float64).reshape(fo, fi)
        off += fi * fo
        b = params[off:off + fo].astype(np.float64)
        off += fo
        c = 16 * -(-fi // 64)  # fan-in chunk
        prod = Wl * a[None, :]
        sq = np.zeros(fo)
        totals = []
        for g in range(0, fi, c):
            partial = np.cumsum(prod[:, g:g + c], axis=1)  # the running sums one fmaf chain rounds
            sq += (partial ** 2).sum(axis=1)
            totals.append(partial[:, -1])
        running = np.cumsum(np.stack(totals), axis=0)  # the chunk sums added in order
        sq += (running[1:] ** 2).sum(axis=0)
        z = running[-1] + b
        v = sq * _U * _U / 3.0 + z * z * _U * _U / 3.0 + (Wl * Wl) @ var
        if l + 1 < L:
            a, slope = _act(w.acts[l], z)
            # FP32 tanh/erf: a few ulps; GELU's 1 + erf loses them relative to
            # the result where erf nears -1, so its error scales with |z| there
            noise = 0.0 if w.acts[l] == W.ACT_RELU else 4.0 * _U * (np.abs(a) + (w.acts[l] == W.ACT_GELU) * np.abs(z))
            var = slope * slope * v + noise ** 2
        else:
            return float(z[0]), math.sqrt(float(v[0]))


def fp32_sigma_rows(w, params, xs, batch=8, n_threads=8):
    """fp32_sigma for many inputs at once (the same model, vectorised over
    rows, batches on host threads): arrays of the FP64 outputs and of the
    error standard deviations."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(n_threads) as ex:
        parts = list(ex.map(lambda r0: _fp32_sigma_batch(w, params, xs[r0:r0 + batch]), range(0, len(xs), batch)))
    return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])


def _fp32_sigma_batch(w, params, xs):
    a = xs.astype(np.float64)
    var = np.zeros_like(a)
    off = 0
    L = len(w.widths) - 1
    for l in range(L):
        fi, fo = w.widths[l], w.widths[l + 1]
        Wl = params[off:off + fi * fo].astype(np.float64).reshape(fo, fi)
        off += fi * fo
        b = params[off:off + fo].astype(np.float64)
        off += fo
        c = 16 * -(-fi // 64)
        prod = Wl[None, :, :] * a[:, None, :]
        sq = np.zeros((a.shape[0], fo))
        totals = []
        for g in range(0, fi, c):
            partial = np.cumsum(prod[:, :, g:g + c], axis=2)
            sq += (partial ** 2).sum(axis=2)
            totals.append(partial[:, :, -1])
        running = np.cumsum(np.stack(totals), axis=0)
        sq += (running[1:] ** 2).sum(axis=0)
        z = running[-1] + b[None, :]
        v = sq * _U * _U / 3.0 + z * z * _U * _U / 3.0 + var @ (Wl * Wl).T
        if l + 1 < L:
            a, slope = _act(w.acts[l], z)
            noise = 0.0 if w.acts[l] == W.ACT_RELU else 4.0 * _U * (np.abs(a) + (w.acts[l] == W.ACT_GELU) * np.abs(z))
            var = slope * slope * v + noise ** 2
    return z[:, 0], np.sqrt(v[:, 0])


def _inputs(w, n, seed):
    rng = np.random.default_rng(seed)
    xs = rng.uniform(w.lb, w.ub, size=(n, w.dim)).astype(np.float32)
    xs[0] = w.lb
    xs[1] = w.ub
    xs[2] = 0.0
    return xs


NETS = [1, 2, 3, 5, 6, 8, 9, 10, 12]


@pytest.mark.parametrize("net_id", NETS)
def test_fitness_matches_oracle(pkg, net_id):
    """Every Table 2 shape: 130 rows (two full tiles and a ragged one), box
    corners and the centre among them."""
    w = W.table2_net(net_id)
    params = W.make_net(w)
    prob = oracle.Problem.for_workload(w)
    xs = _inputs(w, 130, 7 + net_id)
    with pkg.Mgfwa.for_workload(w, 1) as run:
        got = run.evaluate(xs).astype(np.float64)
    ref = prob.fitness_many(xs)
    # the tolerance model on every row (vectorised over rows)
    f64, sig = fp32_sigma_rows(w, params, xs)
    bad = np.abs(f64 - ref) > 1e-9 * np.maximum(1.0, np.abs(ref))
    assert not bad.any(), (net_id, np.nonzero(bad)[0][:8])
    bad = np.abs(got - ref) > 10.0 * sig + 1e-30
    assert not bad.any(), (net_id, [(int(i), got[i], ref[i], sig[i]) for i in np.nonzero(bad)[0][:4]])
    assert np.all(np.abs(got - ref) <= 1e-3 * (np.abs(ref) + 1e-2))


def test_single_linear_layer_and_tanh(pkg):
    """Degenerate shapes: one linear layer (no hidden activation; the
    minimum over the box is b - sum |w_i| at x = -sign(w)) and a tanh stack
    with widths that are multiples of nothing."""
    lin = W.scaled(W.table2_net(1), widths=(10, 1), acts=(), name="lin10")
    params = W.make_net(lin)
    wv, b = params[:10].astype(np.float64), float(params[10])
    xs = _inputs(lin, 67, 3)
    xs[3] = -np.sign(wv).astype(np.float32)
    with pkg.Mgfwa.for_workload(lin, 2) as run:
        got = run.evaluate(xs).astype(np.float64)
    exact = xs.astype(np.float64) @ wv + b
    assert np.all(np.abs(got - exact) <= 1e-6 * (np.abs(xs) @ np.abs(wv) + abs(b)))
    assert abs(got[3] - (b - np.abs(wv).sum())) <= 1e-5

    odd = W.scaled(W.table2_net(3), widths=(20, 13, 77, 5, 1), acts=(W.ACT_TANH,) * 3, name="odd")
    prob = oracle.Problem.for_workload(odd)
    params = W.make_net(odd)
    xs = _inputs(odd, 65, 4)
    with pkg.Mgfwa.for_workload(odd, 3) as run:
        got = run.evaluate(xs).astype(np.float64)
    ref = prob.fitness_many(xs)
    _, sig = fp32_sigma_rows(odd, params, xs)
    bad = np.abs(got - ref) > 10.0 * sig + 1e-30
    assert not bad.any(), [(int(i), got[i], ref[i], sig[i]) for i in np.nonzero(bad)[0][:4]]


def test_maximum_shapes(pkg):
    """The ABI's limits: a 4096-wide layer (GELU) and 16 layers; 70 rows (a full 64-row tile and a
    ragged one)."""
    wide = W.scaled(W.table2_net(2), widths=(4096, 4096, 1), acts=(W.ACT_GELU,), dim=4096, name="wide")
    deep = W.scaled(W.table2_net(1), widths=(10,) + (24,) * 15 + (1,), acts=(W.ACT_RELU,) * 15, name="deep")
    for w, n_model in ((wide, 8), (deep, 70)):
        params = W.make_net(w)
        prob = oracle.Problem.for_workload(w)
        xs = _inputs(w, 70, 21)
        with pkg.Mgfwa.for_workload(w, 4) as run:
            got = run.evaluate(xs).astype(np.float64)
            x0, f0, _ = run.best()  # the FP64 report (64 KB of shared memory at width 4096)
        assert abs(f0 - prob.fitness(x0)) <= 1e-9 * max(1.0, abs(f0)), w.name
        ref = prob.fitness_many(xs, n_threads=8)
        # the tolerance model on the first n_model rows (all of the deep stack's; at width 4096 a row's model
        # is 16M products)
        _, sig = fp32_sigma_rows(w, params, xs[:n_model], batch=1 if w.dim > 1000 else 8)
        bad = np.abs(got[:n_model] - ref[:n_model]) > 10.0 * sig + 1e-30
        assert not bad.any(), (w.name, [(int(i), got[i], ref[i], sig[i]) for i in np.nonzero(bad)[0][:4]])
        assert np.all(np.abs(got - ref) <= 1e-3 * (np.abs(ref) + 1e-2)), w.name


def test_value_does_not_depend_on_the_batch(pkg):
    """A spark's value is the same bit for bit whichever rows share its launch: 1040 rows (64-row tiles
    on the wide layers), 40 at a time and 7 (32-row tiles)."""
    w = W.table2_net(10)
    xs = _inputs(w, 1040, 5)
    with pkg.Mgfwa.for_workload(w, 1) as run:
        full = run.evaluate(xs)
        parts = np.concatenate([run.evaluate(xs[i:i + 40]) for i in range(0, len(xs), 40)])
        few = run.evaluate(xs[100:107])
    assert np.array_equal(full, parts)
    assert np.array_equal(full[100:107], few)


@pytest.mark.parametrize("net_id", [5, 10])
def test_generation_fitness_and_reported_best(pkg, net_id):
    """Whole generations through the library: every spark's fitness (read
    back phase by phase) matches the oracle on the spark the GPU made, the
    reported best (FP64 on the device) matches the oracle's FP64 value of the
    returned vector, and it never rises above the initial fireworks' best."""
    w = W.scaled(W.table2_net(net_id), sparks_per_firework=40, guiding_per_firework=4,
                 eval_budget=W.budget_for_generations(5, 40, 4, 30))
    prob = oracle.Problem.for_workload(w)
    with pkg.Mgfwa.for_workload(w, 11) as run:
        _, f0, _ = run.best()
        for _ in range(2):
            run.phase(pkg.MGFWA_PHASE_EXPLODE)
            run.phase(pkg.MGFWA_PHASE_EVAL_E)
            sp = run.read(pkg.MGFWA_BUF_SPARKS)[:, :w.dim]
            fe = run.read(pkg.MGFWA_BUF_FIT_E).astype(np.float64)
            ref = prob.fitness_many(sp)
            assert np.all(np.abs(fe - ref) <= 1e-4 * (np.abs(ref) + 1e-2))
            for ph in (pkg.MGFWA_PHASE_RANK, pkg.MGFWA_PHASE_GUIDE, pkg.MGFWA_PHASE_EVAL_G):
                run.phase(ph)
            gd = run.read(pkg.MGFWA_BUF_GUIDES)[:, :w.dim]
            fg = run.read(pkg.MGFWA_BUF_FIT_G).astype(np.float64)
            ref = prob.fitness_many(gd)
            assert np.all(np.abs(fg - ref) <= 1e-4 * (np.abs(ref) + 1e-2))
            run.phase(pkg.MGFWA_PHASE_SELECT)
        run.run()
        x, f, ev = run.best()
    assert ev == w.eval_budget
    assert np.all(x >= w.lb) and np.all(x <= w.ub)
    assert abs(f - prob.fitness(x)) <= 1e-9 * max(1.0, abs(f))
    assert f <= f0 + 1e-5 * (1.0 + abs(f0))  # the run keeps its FP32 best; FP64 may reorder near-ties
