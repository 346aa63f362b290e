"""The testbed objective (Sec. 4.1, Eq. 1) with FP32X3: the network's layers
on the tensor cores at FP32 accuracy, against the oracle.

Each layer with fan_in % 8 == 0 and an even fan_out >= 16 runs as six BF16
products per 16-element K step: both operands split into three BF16 parts
(v = v1 + v2 + v3 + r, |r| <= 2^-27 |v|), the products a1b1 into two FP32
accumulators (even and odd 32-element K blocks) and a1b2, a2b1, a2b2,
a1b3, a3b1 into a third, added in the epilogue; the fan-in is cut into
splits of 128 elements whose partial sums are added in split order.  The tolerance follows that
arithmetic: every product carries at most 2^-25 of its magnitude in
dropped parts and residuals, every MMA step rounds its accumulator by at
most one FP32 ulp (2^-23 of the running sum), each epilogue add by half an
ulp; each is modelled as an independent error of that size, propagated in
FP64 through the network's own weights and activation slopes, and the test
allows 10 of the resulting standard deviations (plus a few ulps of tanh and
erf at each activation).  The other layers (here the final 1-output one) are
the CUDA-core layers with their own model (the FP32 test's).  A dropped
product, a missing correction or a wrong index moves the output by far
more."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from test_gpu_net_output import _act, _inputs

pytestmark = pytest.mark.gpu

_U = 2.0 ** -24


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2501_03944_gb300 as p
    return p


def _x3_layer(fi, fo):
    return fi % 8 == 0 and fo >= 16 and fo % 2 == 0


def x3_sigma(w, params, x):
    """FP64 forward of one input and the standard deviation of the FP32X3 forward's error (module docstring)."""
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
        prod = Wl * a[None, :]
        if _x3_layer(fi, fo):
            sq = ((2.0 ** -25 * np.abs(prod)) ** 2).sum(axis=1) / 3.0           # the products' dropped parts
            steps = -(-fi // 16)
            pad = np.zeros((fo, steps * 16))
            pad[:, :fi] = prod
            step_sum = pad.reshape(fo, steps, 16).sum(axis=2)                  # one MMA step's 16 products
            # K splits of 4 blocks (8 steps); in each, the main accumulator of a step alternates by block
            running = np.zeros(fo)
            for s0 in range(0, steps, 8):
                part = step_sum[:, s0:s0 + 8]
                acc = (np.arange(part.shape[1]) // 2) % 2
                totals = []
                for k in (0, 1):
                    partial = np.cumsum(part[:, acc == k], axis=1)
                    sq += ((2.0 * _U * partial) ** 2).sum(axis=1) / 3.0        # one ulp per step
                    totals.append(partial[:, -1] if partial.shape[1] else np.zeros(fo))
                main = totals[0] + totals[1]
                sq += 2.0 * (_U * main) ** 2 / 3.0                             # (even + odd) + corrections
                running = running + main
                if s0 > 0:
                    sq += (_U * running) ** 2 / 3.0                            # the splits added in order
            z = running + b
            sq += (_U * z) ** 2 / 3.0
        else:
            c = 16 * -(-fi // 64)  # the CUDA-core layer's fan-in chunk
            sq = np.zeros(fo)
            totals = []
            for g in range(0, fi, c):
                partial = np.cumsum(prod[:, g:g + c], axis=1)
                sq += (partial ** 2).sum(axis=1) * _U * _U / 3.0
                totals.append(partial[:, -1])
            running = np.cumsum(np.stack(totals), axis=0)
            sq += (running[1:] ** 2).sum(axis=0) * _U * _U / 3.0
            z = running[-1] + b
            sq += z * z * _U * _U / 3.0
        v = sq + (Wl * Wl) @ var
        if l + 1 < L:
            a, slope = _act(w.acts[l], z)
            noise = 0.0 if w.acts[l] == W.ACT_RELU else 4.0 * _U * (np.abs(a) + (w.acts[l] == W.ACT_GELU) * np.abs(z))
            var = slope * slope * v + noise ** 2
        else:
            return float(z[0]), math.sqrt(float(v[0]))


def x3_sigma_rows(w, params, xs, batch=8, n_threads=8):
    """x3_sigma for many inputs at once (the same model, vectorised over rows, batches on host threads):
    arrays of the FP64 outputs and of the error standard deviations."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(n_threads) as ex:
        parts = list(ex.map(lambda r0: _x3_sigma_batch(w, params, xs[r0:r0 + batch]), range(0, len(xs), batch)))
    return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])


def _x3_sigma_batch(w, params, xs):
    a = xs.astype(np.float64)
    R = a.shape[0]
    var = np.zeros_like(a)
    off = 0
    L = len(w.widths) - 1
    for l in range(L):
        fi, fo = w.widths[l], w.widths[l + 1]
        Wl = params[off:off + fi * fo].astype(np.float64).reshape(fo, fi)
        off += fi * fo
        b = params[off:off + fo].astype(np.float64)
        off += fo
        prod = Wl[None, :, :] * a[:, None, :]
        if _x3_layer(fi, fo):
            sq = ((2.0 ** -25 * np.abs(prod)) ** 2).sum(axis=2) / 3.0
            steps = -(-fi // 16)
            pad = np.zeros((R, fo, steps * 16))
            pad[:, :, :fi] = prod
            step_sum = pad.reshape(R, fo, steps, 16).sum(axis=3)
            running = np.zeros((R, fo))
            for s0 in range(0, steps, 8):
                part = step_sum[:, :, s0:s0 + 8]
                acc = (np.arange(part.shape[2]) // 2) % 2
                totals = []
                for k in (0, 1):
                    partial = np.cumsum(part[:, :, acc == k], axis=2)
                    sq += ((2.0 * _U * partial) ** 2).sum(axis=2) / 3.0
                    totals.append(partial[:, :, -1] if partial.shape[2] else np.zeros((R, fo)))
                main = totals[0] + totals[1]
                sq += 2.0 * (_U * main) ** 2 / 3.0
                running = running + main
                if s0 > 0:
                    sq += (_U * running) ** 2 / 3.0
            z = running + b[None, :]
            sq += (_U * z) ** 2 / 3.0
        else:
            c = 16 * -(-fi // 64)
            sq = np.zeros((R, fo))
            totals = []
            for g in range(0, fi, c):
                partial = np.cumsum(prod[:, :, g:g + c], axis=2)
                sq += (partial ** 2).sum(axis=2) * _U * _U / 3.0
                totals.append(partial[:, :, -1])
            running = np.cumsum(np.stack(totals), axis=0)
            sq += (running[1:] ** 2).sum(axis=0) * _U * _U / 3.0
            z = running[-1] + b[None, :]
            sq += z * z * _U * _U / 3.0
        v = sq + var @ (Wl * Wl).T
        if l + 1 < L:
            a, slope = _act(w.acts[l], z)
            noise = 0.0 if w.acts[l] == W.ACT_RELU else 4.0 * _U * (np.abs(a) + (w.acts[l] == W.ACT_GELU) * np.abs(z))
            var = slope * slope * v + noise ** 2
    return z[:, 0], np.sqrt(v[:, 0])


NETS = [2, 3, 5, 6, 8, 9, 10, 12]


@pytest.mark.parametrize("net_id", NETS)
def test_fp32x3_matches_oracle(pkg, net_id):
    """Table 2 shapes with at least one tensor-core layer: 130 rows (a full 128-row tile and a ragged one), box
    corners and the centre among them."""
    w = W.table2_net(net_id)
    params = W.make_net(w)
    prob = oracle.Problem.for_workload(w)
    xs = _inputs(w, 130, 70 + net_id)
    with pkg.Mgfwa.for_workload(w, 1, precision=pkg.MGFWA_FP32X3) as run:
        got = run.evaluate(xs, pkg.MGFWA_FP32X3).astype(np.float64)
        again = run.evaluate(xs, pkg.MGFWA_FP32X3)
        simt = run.evaluate(xs, pkg.MGFWA_FP32).astype(np.float64)
    assert np.array_equal(got.astype(np.float32), again)
    ref = prob.fitness_many(xs)
    # the tolerance model on every row (vectorised over rows)
    f64, sig = x3_sigma_rows(w, params, xs)
    bad = np.abs(f64 - ref) > 1e-9 * np.maximum(1.0, np.abs(ref))
    assert not bad.any(), (net_id, np.nonzero(bad)[0][:8])
    bad = np.abs(got - ref) > 10.0 * sig + 1e-30
    assert not bad.any(), (net_id, [(int(i), got[i], ref[i], sig[i]) for i in np.nonzero(bad)[0][:4]])
    assert np.all(np.abs(got - ref) <= 1e-3 * (np.abs(ref) + 1e-2))
    # the CUDA-core path of the same handle agrees within both paths' errors
    assert np.all(np.abs(got - simt) <= 1e-3 * (np.abs(ref) + 1e-2))


def test_fp32x3_wide_and_deep(pkg):
    """A 4096-wide GELU layer and a 16-layer ReLU stack of width 24 (layers of fan_in 24 % 8 == 0 and fan_out
    24 on the tensor cores, the first of fan_in 10 on the CUDA cores, its output split for the next)."""
    wide = W.scaled(W.table2_net(2), widths=(4096, 4096, 1), acts=(W.ACT_GELU,), dim=4096, name="wide")
    deep = W.scaled(W.table2_net(1), widths=(10,) + (24,) * 15 + (1,), acts=(W.ACT_RELU,) * 15, name="deep")
    for w, n_model in ((wide, 8), (deep, 70)):
        params = W.make_net(w)
        prob = oracle.Problem.for_workload(w)
        xs = _inputs(w, 70, 31)
        with pkg.Mgfwa.for_workload(w, 4, precision=pkg.MGFWA_FP32X3) as run:
            got = run.evaluate(xs, pkg.MGFWA_FP32X3).astype(np.float64)
        ref = prob.fitness_many(xs, n_threads=8)
        _, sig = x3_sigma_rows(w, params, xs[:n_model], batch=1 if w.dim > 1000 else 8)
        bad = np.abs(got[:n_model] - ref[:n_model]) > 10.0 * sig + 1e-30
        assert not bad.any(), (w.name, [(int(i), got[i], ref[i], sig[i]) for i in np.nonzero(bad)[0][:4]])
        assert np.all(np.abs(got - ref) <= 1e-3 * (np.abs(ref) + 1e-2)), w.name


def test_fp32x3_value_does_not_depend_on_the_batch(pkg):
    """Bitwise the same value whichever rows share the launch: 1040 rows, 40 at a time, and 7."""
    w = W.table2_net(10)
    xs = _inputs(w, 1040, 5)
    with pkg.Mgfwa.for_workload(w, 1, precision=pkg.MGFWA_FP32X3) as run:
        full = run.evaluate(xs, pkg.MGFWA_FP32X3)
        parts = np.concatenate([run.evaluate(xs[i:i + 40], pkg.MGFWA_FP32X3) for i in range(0, len(xs), 40)])
        few = run.evaluate(xs[100:107], pkg.MGFWA_FP32X3)
    assert np.array_equal(full, parts)
    assert np.array_equal(full[100:107], few)


def test_fp32x3_generations_and_rejections(pkg):
    """Whole generations in FP32X3: every spark's fitness matches the oracle on the spark the GPU made, the
    reported best is the oracle's FP64 value of the returned vector; FP32X3 is refused for the MLP objective,
    for a network with no qualifying layer, and for evaluation on an FP32 handle."""
    w = W.scaled(W.table2_net(10), sparks_per_firework=40, guiding_per_firework=4,
                 eval_budget=W.budget_for_generations(5, 40, 4, 10))
    prob = oracle.Problem.for_workload(w)
    with pkg.Mgfwa.for_workload(w, 11, precision=pkg.MGFWA_FP32X3) as run:
        for _ in range(2):
            run.phase(pkg.MGFWA_PHASE_EXPLODE)
            run.phase(pkg.MGFWA_PHASE_EVAL_E)
            sp = run.read(pkg.MGFWA_BUF_SPARKS)[:, :w.dim]
            fe = run.read(pkg.MGFWA_BUF_FIT_E).astype(np.float64)
            ref = prob.fitness_many(sp)
            assert np.all(np.abs(fe - ref) <= 1e-4 * (np.abs(ref) + 1e-2))
            for ph in (pkg.MGFWA_PHASE_RANK, pkg.MGFWA_PHASE_GUIDE, pkg.MGFWA_PHASE_EVAL_G, pkg.MGFWA_PHASE_SELECT):
                run.phase(ph)
        run.run()
        x, f, ev = run.best()
    assert ev == w.eval_budget
    assert abs(f - prob.fitness(x)) <= 1e-9 * max(1.0, abs(f))
    mlp = W.scaled(W.MLP_8_16_3, n_samples=64)
    X, y = W.make_data(mlp)
    with pytest.raises(pkg.MgfwaError):
        pkg.Mgfwa.for_workload(mlp, 1, precision=pkg.MGFWA_FP32X3, X=X, y=y)
    tiny = W.scaled(W.table2_net(1), widths=(10, 12, 1), acts=(W.ACT_TANH,), name="tiny")
    with pytest.raises(pkg.MgfwaError):
        pkg.Mgfwa.for_workload(tiny, 1, precision=pkg.MGFWA_FP32X3)
    with pkg.Mgfwa.for_workload(W.table2_net(10), 1) as run:
        with pytest.raises(pkg.MgfwaError):
            run.evaluate(_inputs(W.table2_net(10), 4, 1), pkg.MGFWA_FP32X3)
