"""Groups: many runs of different shapes (dimension, population, network,
batch, precision) stepped together, one CUDA graph launch per generation
(the batching trait for uneven runs), the paper's testbed objective among them.  The claim to check is that grouping
changes no result: every member ends bitwise where the same handle ends
when run alone, also when its budget ends before the others' (the graph is
captured again without it) and when group steps and the member's own steps
alternate."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2501_03944_gb300 as p
    return p


def _specs(pkg):
    small = W.MLP_8_16_3
    big = W.scaled(W.MLP_784_64_10, n_samples=300, n_fireworks=3, sparks_per_firework=20, guiding_per_firework=4)
    deep = W.scaled(W.MLP_784_64_10, widths=(64, 64, 32, 5), acts=(1, 0), n_samples=256, n_fireworks=2,
                    sparks_per_firework=16, guiding_per_firework=4)
    return [
        (W.scaled(small, eval_budget=W.budget_for_generations(5, 40, 4, 15)), 11, pkg.MGFWA_FP32, {}),
        (W.scaled(big, eval_budget=W.budget_for_generations(3, 20, 4, 6)), 12, pkg.MGFWA_BF16, {}),
        (W.scaled(W.SPHERE_30, eval_budget=W.budget_for_generations(5, 40, 4, 8)), 13, pkg.MGFWA_FP32, {}),
        (W.scaled(small, eval_budget=W.budget_for_generations(5, 40, 4, 10)), 14, pkg.MGFWA_FP32, {"n_runs": 2}),
        (W.scaled(deep, eval_budget=W.budget_for_generations(2, 16, 4, 5)), 15, pkg.MGFWA_BF16, {}),
        (W.scaled(big, eval_budget=W.budget_for_generations(3, 20, 4, 4)), 16, pkg.MGFWA_FP8, {"elite_rescore": 0}),
        (W.scaled(W.table2_net(6), sparks_per_firework=40, guiding_per_firework=4,
                  eval_budget=W.budget_for_generations(5, 40, 4, 7)), 17, pkg.MGFWA_FP32, {}),
        # more members on the CTA-pair kernel, so that the group's grouped fitness launches cover several
        # handles: two runs without the re-score (the group finishes their guiding means), and d_in = 96
        # (a partial last K atom) with another batch size
        (W.scaled(big, n_samples=200, eval_budget=W.budget_for_generations(3, 20, 4, 5)), 18, pkg.MGFWA_BF16,
         {"n_runs": 2, "elite_rescore": 0}),
        (W.scaled(big, widths=(96, 64, 10), n_samples=700, eval_budget=W.budget_for_generations(3, 20, 4, 7)), 19,
         pkg.MGFWA_BF16, {}),
    ]


def _make(pkg, w, seed, prec, kw):
    X, y = W.make_data(w) if w.kind == W.KIND_MLP_CE else (None, None)
    return pkg.Mgfwa.for_workload(w, seed, precision=prec, X=X, y=y, **kw)


def _state(pkg, h):
    B = h.cfg.n_runs
    return [h.best(b) for b in range(B)], h.read(pkg.MGFWA_BUF_FW_F), h.info().generations


def _same(a, b):
    (bests_a, fw_a, g_a), (bests_b, fw_b, g_b) = a, b
    assert g_a == g_b and np.array_equal(fw_a, fw_b)
    for (xa, fa, ea), (xb, fb, eb) in zip(bests_a, bests_b):
        assert np.array_equal(xa, xb) and fa == fb and ea == eb


def test_group_members_equal_runs_made_alone(pkg):
    specs = _specs(pkg)
    members = [_make(pkg, *sp) for sp in specs]
    with pkg.Group(members) as g:
        g.run()
        assert g.step(1) == pkg.MGFWA_EBUDGET
    for h, sp in zip(members, specs):
        got = _state(pkg, h)
        h.close()
        with _make(pkg, *sp) as alone:
            alone.run()
            _same(got, _state(pkg, alone))


def test_group_steps_and_own_steps_interleave(pkg):
    specs = _specs(pkg)[:3]
    members = [_make(pkg, *sp) for sp in specs]
    g = pkg.Group(members)
    g.step(2)
    members[0].step(3)          # on the member's own stream, after the group's generations
    g.step(2)
    g.close()
    members[1].step(1)          # usable alone again after the group is gone
    for h, sp, n in zip(members, specs, (7, 5, 4)):
        got = _state(pkg, h)
        h.close()
        with _make(pkg, *sp) as alone:
            alone.step(n)
            _same(got, _state(pkg, alone))


def test_group_rejections(pkg):
    specs = _specs(pkg)
    a = _make(pkg, *specs[0])
    r = _make(pkg, specs[0][0], 1, pkg.MGFWA_FP32, {"refine_every": 2, "refine_steps": 2, "refine_lr": 0.1})
    with pytest.raises(pkg.MgfwaError):
        pkg.Group([a, a])
    with pytest.raises(pkg.MgfwaError):
        pkg.Group([a, r])
    with pkg.Group([a]):
        with pytest.raises(pkg.MgfwaError):
            pkg.Group([a])      # already in a group
    a.close()
    r.close()


def test_mixed_batch_group(pkg):
    """Sixteen runs drawn like the 64-run batching workload (D log-uniform over the MLP families, 3..8 fireworks,
    32..256 sparks, batches of 512..2048), BF16 where the tensor-core path takes the net, FP32 otherwise."""
    ws = W.mixed_batch(16, seed=7, generations=3)
    precs = [pkg.MGFWA_BF16 if w.widths[1] == 64 else pkg.MGFWA_FP32 for w in ws]
    members = [_make(pkg, w, 100 + k, p, {}) for k, (w, p) in enumerate(zip(ws, precs))]
    with pkg.Group(members) as g:
        g.run()
    for k, (h, w, p) in enumerate(zip(members, ws, precs)):
        got = _state(pkg, h)
        h.close()
        with _make(pkg, w, 100 + k, p, {}) as alone:
            alone.run()
            _same(got, _state(pkg, alone))


def test_group_three_layer_pair_members(pkg):
    """Three members on the three-layer CTA-pair kernel (3072-128-64-10): one grouped fitness launch serves
    all of them (batches of 300, 512 and 700 samples; an odd spark count per launch in one, and E4M3 in
    another, which runs on its own branch), and each ends bitwise where it ends alone."""
    base = W.scaled(W.MLP_3072_128_64_10, n_fireworks=2, sparks_per_firework=12, guiding_per_firework=4,
                    eval_budget=W.budget_for_generations(2, 12, 4, 4))
    specs = [
        (W.scaled(base, n_samples=300), 41, pkg.MGFWA_BF16, {}),
        (W.scaled(base, n_samples=512, n_fireworks=3, sparks_per_firework=8,
                  eval_budget=W.budget_for_generations(3, 8, 4, 3)), 42, pkg.MGFWA_BF16, {"elite_rescore": 0}),
        (W.scaled(base, n_samples=700), 43, pkg.MGFWA_BF16, {"n_runs": 2}),
        (W.scaled(base, n_samples=512), 44, pkg.MGFWA_FP8, {"elite_rescore": 0}),
    ]
    members = [_make(pkg, *sp) for sp in specs]
    with pkg.Group(members) as g:
        g.run()
    for h, sp in zip(members, specs):
        got = _state(pkg, h)
        h.close()
        with _make(pkg, *sp) as alone:
            alone.run()
            _same(got, _state(pkg, alone))
