"""B independent runs per handle: the batch dimension of GPU-MGFWA (Sec. 3,
Table 1: every variable gets a leading batch dimension B).

Run b of a handle seeded s is the single run seeded s + b: every run is
checked phase by phase against the oracle run with that seed (bit-exact
positions, ranks and selection when fed the oracle's fitness), and a batch
of runs gives bitwise the same results as the same runs made one by one --
in FP32 and on the tensor-core path, whose per-spark sums do not depend on
which sparks share a tile.
"""
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


def _rel(a, b, rtol, atol):
    return np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)) / (np.abs(b) + atol / rtol)


def test_each_run_follows_its_oracle_run(pkg):
    B = 3
    w = W.scaled(W.MLP_8_16_3, n_samples=200, n_fireworks=3, sparks_per_firework=12, guiding_per_firework=3)
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    p = oracle.params_for(w)
    seed = 40
    mu, lam, m, D = w.n_fireworks, w.sparks_per_firework, w.guiding_per_firework, w.dim
    with pkg.Mgfwa.for_workload(w, seed, X=X, y=y, n_runs=B) as run:
        st = [oracle.init(p, seed + b) for b in range(B)]
        fx = run.read(pkg.MGFWA_BUF_FW_X).reshape(B, mu, D)
        for b in range(B):
            assert np.array_equal(fx[b], st[b][0])
        f0 = [prob.fitness_many(st[b][0]).astype(np.float32) for b in range(B)]
        run.write(pkg.MGFWA_BUF_FW_F, np.concatenate(f0))
        state = [(st[b][0], st[b][1], f0[b]) for b in range(B)]
        for gen in (1, 2):
            refs = [oracle.generation(p, prob, seed + b, gen, *state[b]) for b in range(B)]
            run.phase(pkg.MGFWA_PHASE_EXPLODE)
            sp = run.read(pkg.MGFWA_BUF_SPARKS).reshape(B, mu * lam, D)
            for b in range(B):
                assert np.array_equal(sp[b], refs[b]["sparks"]), (gen, b)
            run.phase(pkg.MGFWA_PHASE_EVAL_E)
            fe = run.read(pkg.MGFWA_BUF_FIT_E).reshape(B, -1)
            for b in range(B):
                assert np.all(_rel(fe[b], refs[b]["fit_e64"], 1e-5, 1e-5) <= 1e-5)
            run.write(pkg.MGFWA_BUF_FIT_E, np.concatenate([r["fit_e"] for r in refs]))
            run.phase(pkg.MGFWA_PHASE_RANK)
            top = run.read(pkg.MGFWA_BUF_TOP).reshape(B, mu, m, -1)
            for b in range(B):
                assert np.array_equal(top[b], refs[b]["top"])
            run.phase(pkg.MGFWA_PHASE_GUIDE)
            gd = run.read(pkg.MGFWA_BUF_GUIDES).reshape(B, mu * m, D)
            for b in range(B):
                assert np.array_equal(gd[b], refs[b]["guides"]), (gen, b)
            run.phase(pkg.MGFWA_PHASE_EVAL_G)
            run.write(pkg.MGFWA_BUF_FIT_G, np.concatenate([r["fit_g"] for r in refs]))
            run.phase(pkg.MGFWA_PHASE_SELECT)
            fx = run.read(pkg.MGFWA_BUF_FW_X).reshape(B, mu, D)
            fa = run.read(pkg.MGFWA_BUF_FW_AMP).reshape(B, mu)
            for b in range(B):
                assert np.array_equal(fx[b], refs[b]["fw_x"]) and np.array_equal(fa[b], refs[b]["fw_amp"])
            state = [(r["fw_x"], r["fw_amp"], r["fw_f"]) for r in refs]
        assert run.info().n_runs == B and run.info().sparks_per_gen == B * w.sparks_per_generation


@pytest.mark.parametrize("precision,w", [
    ("fp32", W.scaled(W.MLP_8_16_3, eval_budget=5 + 12 * 220)),
    ("bf16", W.scaled(W.MLP_784_64_10, n_samples=300, n_fireworks=3, sparks_per_firework=20, guiding_per_firework=4,
                      eval_budget=W.budget_for_generations(3, 20, 4, 6))),
])
def test_batch_equals_runs_made_alone(pkg, precision, w):
    prec = {"fp32": pkg.MGFWA_FP32, "bf16": pkg.MGFWA_BF16}[precision]
    B, seed = 4, 123
    X, y = W.make_data(w)
    with pkg.Mgfwa.for_workload(w, seed, precision=prec, X=X, y=y, n_runs=B) as run:
        run.run()
        batched = [run.best(b) for b in range(B)]
        overall = run.best()
        fw_f = run.read(pkg.MGFWA_BUF_FW_F)
    alone = []
    for b in range(B):
        with pkg.Mgfwa.for_workload(w, seed + b, precision=prec, X=X, y=y) as r1:
            r1.run()
            alone.append(r1.best())
            assert np.array_equal(r1.read(pkg.MGFWA_BUF_FW_F), fw_f[b * w.n_fireworks:(b + 1) * w.n_fireworks])
    for (bx, bf, ev), (ax, af, aev) in zip(batched, alone):
        assert np.array_equal(bx, ax) and bf == af and ev == aev
    best_b = min(range(B), key=lambda b: batched[b][1])
    assert overall[1] == batched[best_b][1]
