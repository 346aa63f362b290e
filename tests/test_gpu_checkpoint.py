"""Checkpoint / resume: a run saved after some generations and loaded into a
fresh handle of the same problem continues bitwise as the uninterrupted run
(FP32, BF16 with the elite re-score, several runs per handle, refinement
crossing the resume point), a larger budget may be given on resume, and a
checkpoint is refused by a handle of another problem."""
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


CASES = [
    ("fp32", W.scaled(W.MLP_8_16_3, eval_budget=W.budget_for_generations(5, 40, 4, 9)), {}),
    ("bf16", W.scaled(W.MLP_784_64_10, n_samples=300, n_fireworks=3, sparks_per_firework=20, guiding_per_firework=4,
                      eval_budget=W.budget_for_generations(3, 20, 4, 9)), {"n_runs": 2}),
    ("fp32", W.scaled(W.MLP_8_16_3, eval_budget=W.budget_for_generations(5, 40, 4, 9) + 3 * 7),
     {"refine_every": 3, "refine_steps": 2, "refine_lr": 0.3}),
]


def _state(pkg, h):
    return ([h.best(b) for b in range(h.cfg.n_runs)], h.read(pkg.MGFWA_BUF_FW_X), h.read(pkg.MGFWA_BUF_FW_AMP),
            h.read(pkg.MGFWA_BUF_FW_F), h.info().evals, h.info().generations)


@pytest.mark.parametrize("prec,w,kw", CASES)
def test_resume_continues_the_run(pkg, prec, w, kw):
    p = {"fp32": pkg.MGFWA_FP32, "bf16": pkg.MGFWA_BF16}[prec]
    X, y = W.make_data(w)
    with pkg.Mgfwa.for_workload(w, 21, precision=p, X=X, y=y, **kw) as a:
        a.run()
        want = _state(pkg, a)
    with pkg.Mgfwa.for_workload(w, 21, precision=p, X=X, y=y, **kw) as b:
        b.step(4)
        ck = b.checkpoint()
    with pkg.Mgfwa.for_workload(w, 21, precision=p, X=X, y=y, **kw) as c:
        c.restore(ck)
        assert c.info().generations == 4
        c.run()
        got = _state(pkg, c)
    for (xa, fa, ea), (xb, fb, eb) in zip(want[0], got[0]):
        assert np.array_equal(xa, xb) and fa == fb and ea == eb
    for u, v in zip(want[1:], got[1:]):
        assert np.array_equal(u, v)


def test_resume_with_a_larger_budget_and_refusals(pkg):
    w = W.scaled(W.MLP_8_16_3, eval_budget=W.budget_for_generations(5, 40, 4, 6))
    X, y = W.make_data(w)
    with pkg.Mgfwa.for_workload(w, 3, X=X, y=y) as a:
        a.run()
        ck = a.checkpoint()
    longer = W.scaled(w, eval_budget=W.budget_for_generations(5, 40, 4, 10))
    with pkg.Mgfwa.for_workload(longer, 3, X=X, y=y) as b:
        b.restore(ck)
        b.run()
        assert b.info().generations == 10
        got = b.best()
    with pkg.Mgfwa.for_workload(longer, 3, X=X, y=y) as ref:
        ref.run()
        want = ref.best()
    assert np.array_equal(got[0], want[0]) and got[1] == want[1]
    for other in (W.scaled(w, sigma=0.3), W.scaled(w, n_fireworks=4)):
        with pkg.Mgfwa.for_workload(other, 3, X=X, y=y) as h:
            with pytest.raises(pkg.MgfwaError):
                h.restore(ck)
    with pkg.Mgfwa.for_workload(w, 4, X=X, y=y) as h:   # another seed is another problem
        with pytest.raises(pkg.MgfwaError):
            h.restore(ck)
    X2 = X.copy()
    X2[0, 0] += 1.0
    with pkg.Mgfwa.for_workload(w, 3, X=X2, y=y) as h:  # another batch
        with pytest.raises(pkg.MgfwaError):
            h.restore(ck)
