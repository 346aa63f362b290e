"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test ties one oracle function to something independent of it: a library
routine (triton's Philox4x32-10 run by its CPU interpreter, torch's float64
cross_entropy/linear), a closed form, a distribution law, or brute force on
tiny inputs.  A dropped term, a flipped sign, a wrong index or a transposed
operand anywhere in the oracle fails at least one of them.
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# ---------------------------------------------------------------------------
# Philox4x32-10: the oracle's generator against triton's (a library routine,
# run on the CPU by triton's interpreter in a child process).

_TRITON_PHILOX = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def _k(out_ptr, c0_ptr, c1_ptr, c2_ptr, c3_ptr, seed, n: tl.constexpr):
    i = tl.arange(0, n)
    c0 = tl.load(c0_ptr + i).to(tl.uint32, bitcast=True)
    c1 = tl.load(c1_ptr + i).to(tl.uint32, bitcast=True)
    c2 = tl.load(c2_ptr + i).to(tl.uint32, bitcast=True)
    c3 = tl.load(c3_ptr + i).to(tl.uint32, bitcast=True)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + i * 4 + 0, a.to(tl.int32, bitcast=True))
    tl.store(out_ptr + i * 4 + 1, b.to(tl.int32, bitcast=True))
    tl.store(out_ptr + i * 4 + 2, c.to(tl.int32, bitcast=True))
    tl.store(out_ptr + i * 4 + 3, d.to(tl.int32, bitcast=True))

req = json.loads(sys.stdin.read())
res = []
for seed, ctrs in req:
    ctrs = np.array(ctrs, dtype=np.uint32).reshape(-1, 4)
    n = ctrs.shape[0]
    cols = [torch.from_numpy(ctrs[:, j].astype(np.uint32).view(np.int32).copy()) for j in range(4)]
    out = torch.zeros(4 * n, dtype=torch.int32)
    _k[(1,)](out, *cols, seed, n)
    res.append((out.numpy().view(np.uint32)).tolist())
print(json.dumps(res))
"""


def _triton_philox(requests):
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", _TRITON_PHILOX], input=json.dumps(requests),
                       capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        if "No module named 'triton'" in r.stderr:
            pytest.skip("triton is not installed")
        raise AssertionError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_philox_matches_triton(orc):
    rng = np.random.default_rng(7)
    seeds = [0, 1, 0xDEADBEEF, (0x12345678 << 32) | 0x9ABCDEF0, 2**64 - 1]
    reqs = []
    for s in seeds:
        ctrs = rng.integers(0, 2**32, size=(16, 4), dtype=np.uint64)
        ctrs[0] = 0
        ctrs[1] = [0xFFFFFFFF] * 4
        reqs.append((s, ctrs.astype(np.uint32).ravel().tolist()))
    got_lib = _triton_philox(reqs)
    for (s, flat), lib_out in zip(reqs, got_lib):
        ctrs = np.array(flat, dtype=np.uint32).reshape(-1, 4)
        lib_out = np.array(lib_out, dtype=np.uint32).reshape(-1, 4)
        key = [s & 0xFFFFFFFF, s >> 32]
        for c, want in zip(ctrs, lib_out):
            assert orc.philox(c, key).tolist() == want.tolist()


def test_uniform_counter_layout_against_triton(orc):
    """u(coord) = (lane word >> 8) 2^-24 of Philox(coord/4, unit, gen, purpose) keyed by the seed."""
    seed = (3 << 32) | 11
    picks = [(1, 5, 7, c) for c in range(0, 12)] + [(2, 9, 1, 50889), (3, 0, 200, 402249), (0, 4, 0, 3),
                                                 (1, 2**31, 2047, 402251)]
    reqs = [(seed, [v for (pur, gen, unit, c) in picks for v in (c // 4, unit, gen, pur)])]
    words = np.array(_triton_philox(reqs)[0], dtype=np.uint32).reshape(-1, 4)
    for (pur, gen, unit, c), w in zip(picks, words):
        want = float(np.float32(int(w[c % 4]) >> 8) * np.float32(2.0 ** -24))
        assert orc.uniform(seed, pur, gen, unit, c) == want


# ---------------------------------------------------------------------------
# Uniform draws and initialisation.

def test_init_uniform_and_in_bounds(orc):
    p = orc.make_params(dim=250_000, lb=0.0, ub=1.0, mu=4, lam=8, m=2)
    x, a = orc.init(p, 123)
    u = x.ravel().astype(np.float64)
    assert np.all(u >= 0.0) and np.all(u < 1.0)
    # on the 2^-24 grid
    assert np.all(np.floor(u * 2**24) == u * 2**24)
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    # the four lanes of one Philox block are not copies of each other
    lanes = x.reshape(4, -1, 4)
    assert abs(np.corrcoef(lanes[..., 0].ravel(), lanes[..., 1].ravel())[0, 1]) < 0.01
    assert np.all(a == np.float32(1.0))
    p2 = orc.make_params(dim=1000, lb=-5.0, ub=5.0, mu=3, lam=8, m=2)
    x2, a2 = orc.init(p2, 9)
    assert x2.min() >= -5.0 and x2.max() <= 5.0 and np.all(a2 == np.float32(10.0))
    assert stats.kstest((x2.ravel() + 5.0) / 10.0, "uniform").pvalue > 1e-3


# ---------------------------------------------------------------------------
# Explosion sampling and random mapping.

def test_explosion_counts_and_box_invariant(orc):
    p = orc.make_params(dim=333, lb=-1.0, ub=1.0, mu=4, lam=24, m=4)
    rng = np.random.default_rng(0)
    fw_x = rng.uniform(-1, 1, size=(4, 333)).astype(np.float32)
    fw_x[0, :50] = -1.0
    fw_x[1, :50] = 1.0
    fw_a = np.array([0.3, 0.05, 1.7, 0.0], np.float32)
    s = orc.explode(p, 5, 3, fw_x, fw_a)
    assert s.shape == (4 * 24, 333)
    s3 = s.reshape(4, 24, 333)
    lo = np.maximum(np.float32(-1), fw_x - fw_a[:, None])[:, None, :]
    hi = np.minimum(np.float32(1), fw_x + fw_a[:, None])[:, None, :]
    assert np.all(s3 >= lo) and np.all(s3 <= hi)
    # zero amplitude gives the firework itself
    assert np.all(s3[3] == fw_x[3][None, :])


def test_explosion_is_uniform_in_the_amplitude_box(orc):
    D = 4000
    p = orc.make_params(dim=D, lb=-10.0, ub=10.0, mu=1, lam=64, m=4)
    fw_x = np.zeros((1, D), np.float32)
    fw_a = np.array([0.5], np.float32)
    s = orc.explode(p, 77, 1, fw_x, fw_a)
    t = (s.astype(np.float64) / 0.5).ravel()
    assert t.min() >= -1.0 and t.max() < 1.0
    assert stats.kstest((t + 1.0) / 2.0, "uniform").pvalue > 1e-3


def test_mapping_is_uniform_in_the_clipped_box(orc):
    D = 4000
    p = orc.make_params(dim=D, lb=-1.0, ub=1.0, mu=1, lam=64, m=4)
    fw_x = np.full((1, D), -1.0, np.float32)     # on the lower bound
    fw_a = np.array([0.5], np.float32)
    s = orc.explode(p, 78, 2, fw_x, fw_a)
    v = s.astype(np.float64).ravel()
    assert v.min() >= -1.0 and v.max() <= -0.5
    # half the draws land outside and are redrawn in [lb, x + A]: the mix is uniform there
    assert stats.kstest((v + 1.0) / 0.5, "uniform").pvalue > 1e-3


# ---------------------------------------------------------------------------
# Fitness (FP64 objective).

def _rand_mlp(widths, seed, scale=0.5):
    rng = np.random.default_rng(seed)
    D = W.mlp_param_count(widths)
    return rng.uniform(-scale, scale, size=D).astype(np.float32)


def test_zero_weights_give_log_c(orc):
    for widths, acts in (((8, 16, 3), (orc.TANH,)), ((784, 64, 10), (orc.RELU,)),
                         ((30, 12, 7, 5), (orc.RELU, orc.TANH))):
        rng = np.random.default_rng(1)
        X = rng.normal(size=(37, widths[0])).astype(np.float32)
        y = (np.arange(37) % widths[-1]).astype(np.int32)
        prob = orc.Problem(orc.MLP_CE, W.mlp_param_count(widths), widths, acts, X, y)
        f = prob.fitness(np.zeros(W.mlp_param_count(widths), np.float32))
        assert abs(f - math.log(widths[-1])) < 1e-14


def test_output_bias_closed_form(orc):
    """W = 0 everywhere, hidden bias 0, output bias (t, 0, 0): CE = log(e^t + 2) - t * n0 / N."""
    widths = (8, 16, 3)
    N = 100
    rng = np.random.default_rng(2)
    X = rng.normal(size=(N, 8)).astype(np.float32)
    y = (np.arange(N) % 3).astype(np.int32)
    prob = orc.Problem(orc.MLP_CE, W.mlp_param_count(widths), widths, (orc.RELU,), X, y)
    x = np.zeros(W.mlp_param_count(widths), np.float32)
    t = 2.5
    x[-3] = t
    n0 = int(np.sum(y == 0))
    want = math.log(math.exp(t) + 2.0) - t * n0 / N
    assert abs(prob.fitness(x) - want) < 1e-14


@pytest.mark.parametrize("widths,acts", [((8, 16, 3), ("tanh",)), ((20, 9, 4), ("relu",)),
                                         ((24, 16, 8, 5), ("relu", "relu")),
                                         ((12, 10, 6, 3), ("tanh", "relu"))])
def test_mlp_ce_matches_torch_float64(orc, widths, acts):
    import torch
    import torch.nn.functional as F
    codes = tuple(orc.TANH if a == "tanh" else orc.RELU for a in acts)
    rng = np.random.default_rng(3)
    N = 65
    X = rng.normal(size=(N, widths[0])).astype(np.float32)
    y = (np.arange(N) % widths[-1]).astype(np.int32)
    prob = orc.Problem(orc.MLP_CE, W.mlp_param_count(widths), widths, codes, X, y)
    for seed in range(3):
        x = _rand_mlp(widths, 10 + seed, scale=1.0)
        h = torch.from_numpy(X.astype(np.float64))
        off = 0
        for l in range(len(widths) - 1):
            fi, fo = widths[l], widths[l + 1]
            Wt = torch.from_numpy(x[off:off + fi * fo].astype(np.float64)).reshape(fo, fi)
            off += fi * fo
            b = torch.from_numpy(x[off:off + fo].astype(np.float64))
            off += fo
            h = F.linear(h, Wt, b)
            if l + 1 < len(widths) - 1:
                h = torch.tanh(h) if acts[l] == "tanh" else torch.relu(h)
        want = F.cross_entropy(h, torch.from_numpy(y.astype(np.int64))).item()
        got = prob.fitness(x)
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want))


def test_sphere_value(orc):
    x = np.arange(-7, 23, dtype=np.float32) * np.float32(0.25)
    prob = orc.Problem(orc.SPHERE, 30)
    assert prob.fitness(x) == float(np.sum(x.astype(np.float64) ** 2))


def test_fitness_many_threads_agree(orc):
    w = W.scaled(W.MLP_784_64_10, widths=(784, 8, 10), n_samples=64)
    X, y = W.make_data(w)
    prob = orc.Problem.for_workload(w, X, y)
    xs = W.random_vectors(13, w.dim, -1, 1, 4)
    a = prob.fitness_many(xs, 1)
    b = prob.fitness_many(xs, 4)
    assert np.array_equal(a, b)
    assert a[5] == prob.fitness(xs[5])


# ---------------------------------------------------------------------------
# Ranking: brute force with ties and NaN.

def test_rank_brute_force(orc):
    rng = np.random.default_rng(4)
    for trial in range(40):
        m = int(rng.integers(1, 4))
        g = int(rng.integers(2, 9))
        lam = m * g
        mu = int(rng.integers(1, 4))
        k = int(rng.integers(1, g // 2 + 1))
        p = orc.make_params(dim=1, lb=-1, ub=1, mu=mu, lam=lam, m=m, k=k)
        f = rng.integers(0, 4, size=mu * lam).astype(np.float32)   # many ties
        if trial % 5 == 0:
            f[rng.integers(0, mu * lam)] = np.nan
        top, bot = orc.rank(p, f)
        for i in range(mu):
            for q in range(m):
                idx = list(range(q * g, (q + 1) * g))
                keyf = lambda j: (math.inf if math.isnan(f[i * lam + j]) else float(f[i * lam + j]), j)
                order = sorted(idx, key=keyf)
                assert top[i, q].tolist() == order[:k]
                assert bot[i, q].tolist() == order[::-1][:k]


def test_subset_size(orc):
    assert orc.subset_size(0.2, 10) == 2
    assert orc.subset_size(0.2, 25) == 5
    assert orc.subset_size(0.2, 32) == 6
    assert orc.subset_size(0.5, 4) == 2
    assert orc.subset_size(0.9, 6) == 3      # clamped to g / 2
    assert orc.subset_size(0.01, 8) == 1     # clamped to 1


# ---------------------------------------------------------------------------
# Guiding sparks.

def test_guide_closed_form_linear_ladder(orc):
    """Sparks x + (j+1) d with fitness j: GV = -(g - k) d per coordinate, exactly."""
    mu, m, g, k, D = 2, 3, 8, 3, 17
    lam = m * g
    p = orc.make_params(dim=D, lb=-100, ub=100, mu=mu, lam=lam, m=m, k=k, beta=1.0)
    d = np.float32(2.0 ** -6)
    fw_x = np.zeros((mu, D), np.float32)
    fw_x[1] = 1.5
    fw_a = np.array([50.0, 50.0], np.float32)
    sparks = np.zeros((mu * lam, D), np.float32)
    fit = np.zeros(mu * lam, np.float32)
    for i in range(mu):
        for j in range(lam):
            r = j % g
            sparks[i * lam + j] = fw_x[i] + np.float32((r + 1) * d)
            fit[i * lam + j] = r
    top, bot = orc.rank(p, fit)
    G = orc.guide(p, 1, 1, fw_x, fw_a, sparks, top, bot).reshape(mu, m, D)
    for i in range(mu):
        assert np.all(G[i] == fw_x[i] - np.float32((g - k) * d))
    # with the boost, the same vector scaled
    p2 = orc.make_params(dim=D, lb=-100, ub=100, mu=mu, lam=lam, m=m, k=k, beta=2.0)
    G2 = orc.guide(p2, 1, 1, fw_x, fw_a, sparks, top, bot).reshape(mu, m, D)
    assert np.all(G2[0] == -np.float32(2 * (g - k) * d))


def test_guide_single_group_is_the_gfwa_guiding_spark(orc):
    """m = 1: G = x + (mean of the sigma*lambda best - mean of the sigma*lambda worst)."""
    D, lam = 257, 20
    p = orc.make_params(dim=D, lb=-5, ub=5, mu=1, lam=lam, m=1, sigma=0.2, beta=1.0)
    assert p.k == 4
    rng = np.random.default_rng(5)
    fw_x = rng.uniform(-1, 1, size=(1, D)).astype(np.float32)
    sparks = (fw_x + rng.uniform(-0.5, 0.5, size=(lam, D))).astype(np.float32)
    fit = rng.permutation(lam).astype(np.float32)
    top, bot = orc.rank(p, fit)
    G = orc.guide(p, 2, 1, fw_x, np.array([4.0], np.float32), sparks, top, bot)
    order = np.argsort(fit)
    s64 = sparks.astype(np.float64)
    gv = s64[order[:4]].mean(0) - s64[order[-4:]].mean(0)
    want = fw_x[0].astype(np.float64) + gv
    # FP32 sums of four terms, one divide, one fma: a few ulps of the operands
    assert np.max(np.abs(G[0] - want)) < 8 * np.finfo(np.float32).eps * 2.0


def test_guide_equal_fitness_uses_index_order(orc):
    D, m, g, k = 5, 2, 6, 2
    p = orc.make_params(dim=D, lb=-10, ub=10, mu=1, lam=m * g, m=m, k=k)
    top, bot = orc.rank(p, np.zeros(m * g, np.float32))
    assert top[0].tolist() == [[0, 1], [6, 7]]
    assert bot[0].tolist() == [[5, 4], [11, 10]]


def test_guide_mapping_stays_in_box(orc):
    D, lam, m = 300, 16, 2
    p = orc.make_params(dim=D, lb=-1, ub=1, mu=1, lam=lam, m=m, k=2, beta=8.0)
    rng = np.random.default_rng(6)
    fw_x = rng.uniform(-1, 1, size=(1, D)).astype(np.float32)
    amp = np.array([0.4], np.float32)
    sparks = orc.explode(p, 3, 1, fw_x, amp)
    top, bot = orc.rank(p, rng.permutation(lam).astype(np.float32))
    G = orc.guide(p, 3, 1, fw_x, amp, sparks, top, bot)
    assert np.all(G >= -1) and np.all(G <= 1)
    lo = np.maximum(np.float32(-1), fw_x - amp)
    hi = np.minimum(np.float32(1), fw_x + amp)
    outside = (G < lo) | (G > hi)
    # only unmapped (in-bounds) coordinates may leave the amplitude box
    assert np.all(~outside | ((G >= -1) & (G <= 1)))


# ---------------------------------------------------------------------------
# Selection and amplitude.

def test_select_brute_force(orc):
    rng = np.random.default_rng(8)
    for trial in range(40):
        mu, lam, m, D = 3, 6, 2, 4
        p = orc.make_params(dim=D, lb=-1, ub=1, mu=mu, lam=lam, m=m, k=1, c_a=1.25, c_r=0.5)
        fe = rng.integers(0, 5, size=mu * lam).astype(np.float32)
        fg = rng.integers(0, 5, size=mu * m).astype(np.float32)
        ff = rng.integers(0, 6, size=mu).astype(np.float32)
        if trial % 7 == 0:
            fe[0] = np.nan
        sparks = rng.normal(size=(mu * lam, D)).astype(np.float32)
        guides = rng.normal(size=(mu * m, D)).astype(np.float32)
        fw_x = rng.normal(size=(mu, D)).astype(np.float32)
        fw_a = np.float32(0.25) * np.ones(mu, np.float32)
        nx, na, nf, win = orc.select(p, fe, fg, sparks, guides, fw_x, fw_a, ff)
        for i in range(mu):
            cand = [(math.inf if math.isnan(v) else float(v), c) for c, v in
                    enumerate(list(fe[i * lam:(i + 1) * lam]) + list(fg[i * m:(i + 1) * m]))]
            bf, bc = min(cand)
            if bf < ff[i]:
                assert win[i] == bc and nf[i] == bf and na[i] == np.float32(0.3125)
                row = sparks[i * lam + bc] if bc < lam else guides[i * m + bc - lam]
                assert np.array_equal(nx[i], row)
            else:
                assert win[i] == -1 and nf[i] == ff[i] and na[i] == np.float32(0.125)
                assert np.array_equal(nx[i], fw_x[i])


def test_amplitude_follows_improvement_log(orc):
    w = W.SPHERE_30
    p = orc.params_for(w)
    prob = orc.Problem.for_workload(w)
    fw_x, fw_a = orc.init(p, 4)
    fw_f = prob.fitness_many(fw_x).astype(np.float32)
    a = np.zeros(p.mu, np.int64)
    b = np.zeros(p.mu, np.int64)
    for gen in range(1, 31):
        out = orc.generation(p, prob, 4, gen, fw_x, fw_a, fw_f)
        a += out["winner"] >= 0
        b += out["winner"] < 0
        fw_x, fw_a, fw_f = out["fw_x"], out["fw_amp"], out["fw_f"]
    want = np.float64(p.amp0) * 1.2 ** a * 0.9 ** b
    assert np.allclose(fw_a, want, rtol=1e-5)
    assert a.sum() > 0 and b.sum() > 0


# ---------------------------------------------------------------------------
# Whole runs.

def test_budget_counting(orc):
    w = W.MLP_8_16_3
    p = orc.params_for(w)
    prob = orc.Problem.for_workload(w)
    r = orc.run(p, prob, 0, 1000)
    per = w.sparks_per_generation
    assert r["evals"] == w.n_fireworks + r["gens"] * per
    assert r["evals"] <= 1000 < r["evals"] + per
    r0 = orc.run(p, prob, 0, w.n_fireworks)
    assert r0["gens"] == 0 and r0["evals"] == w.n_fireworks


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sphere_converges_to_zero(orc, seed):
    w = W.SPHERE_30
    r = orc.run(orc.params_for(w), orc.Problem.for_workload(w), seed, w.eval_budget, want_trace=True)
    assert r["evals"] <= 100_000
    assert r["best_f"] < 1e-6
    assert np.all(np.diff(r["trace"]) <= 0)       # best-so-far never worsens


def test_small_mlp_run_learns(orc):
    w = W.MLP_8_16_3
    prob = orc.Problem.for_workload(w)
    p = orc.params_for(w)
    fw_x, _ = orc.init(p, 3)
    start = prob.fitness_many(fw_x).min()
    r = orc.run(p, prob, 3, w.eval_budget, n_threads=4, want_trace=True)
    assert r["evals"] == 19_805 and r["gens"] == 90
    assert r["best_f"] < 0.1 * start and r["best_f"] < math.log(3)
    assert abs(r["best_f"] - r["trace"][-1]) <= 1e-6 * max(1.0, r["best_f"])


def test_table2_parameter_counts():
    """Table 2 of the paper: parameter counts of the testbed nets."""
    path = os.path.join(ROOT, "tests", "golden", "table2_params.json")
    table = json.load(open(path))
    matched = 0
    for net in table["nets"]:
        widths = [net["input"]] + [net["hidden"]] * (net["layer_num"] + 1) + [net["output"]]
        if W.mlp_param_count(widths) == net["params"]:
            matched += 1
            assert net["id"] in table["consistent_ids"]
        else:
            assert net["id"] not in table["consistent_ids"]
    assert matched == len(table["consistent_ids"])
