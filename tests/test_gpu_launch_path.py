"""The launch path changes no result.  A handle replays one captured CUDA
graph per generation (explode .. select), its kernels chained by
programmatic dependent launch; while kernel groups are timed
(mgfwa_debug_profile) it launches the same kernels one by one between
events, and with the fitness means finished by their own kernel instead
of inside the rank and the elite pick.  Both paths must end bitwise in the
same state: FP32, BF16 with the elite re-score (at full size on the
tensor-core FP32 layer with its fused output layer), FP8, a three-layer
net, the sphere, two runs in one handle, the hybrid refinement, the
loser-out tournament and lagged multi-guiding (its first generation kernel
by kernel, the graph from the second)."""
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
    full = W.MLP_784_64_10  # 1040 sparks x 2048 samples; re-score of 10 rows on the tensor-core layer
    return {
        "fp32": (W.scaled(small, eval_budget=W.budget_for_generations(5, 40, 4, 12)), 21, pkg.MGFWA_FP32, {}),
        "bf16": (W.scaled(big, eval_budget=W.budget_for_generations(3, 20, 4, 6)), 22, pkg.MGFWA_BF16, {}),
        "bf16_full": (W.scaled(full, eval_budget=W.budget_for_generations(5, 200, 8, 4)), 23, pkg.MGFWA_BF16, {}),
        "fp8": (W.scaled(big, eval_budget=W.budget_for_generations(3, 20, 4, 5)), 24, pkg.MGFWA_FP8, {}),
        "three_layer": (W.scaled(deep, eval_budget=W.budget_for_generations(2, 16, 4, 5)), 25, pkg.MGFWA_BF16, {}),
        "sphere": (W.scaled(W.SPHERE_30, eval_budget=W.budget_for_generations(5, 40, 4, 8)), 26, pkg.MGFWA_FP32, {}),
        "two_runs": (W.scaled(small, eval_budget=W.budget_for_generations(5, 40, 4, 10)), 27, pkg.MGFWA_FP32,
                     {"n_runs": 2}),
        "refine": (W.scaled(small, eval_budget=3000), 28, pkg.MGFWA_FP32,
                   {"refine_every": 2, "refine_steps": 4, "refine_lr": 0.5}),
        "loser_out": (W.scaled(big, eval_budget=W.budget_for_generations(3, 20, 4, 6)), 29, pkg.MGFWA_BF16,
                      {"loser_out": 1}),
        "lagged_bf16": (W.scaled(big, eval_budget=W.budget_for_generations(3, 20, 4, 6)), 30, pkg.MGFWA_BF16,
                        {"lagged_guiding": 1}),
        "lagged_fp32": (W.scaled(small, eval_budget=W.budget_for_generations(5, 40, 4, 8)), 31, pkg.MGFWA_FP32,
                        {"lagged_guiding": 1}),
        "lagged_two_runs_loser_out": (W.scaled(big, eval_budget=W.budget_for_generations(3, 20, 4, 6)), 32,
                                      pkg.MGFWA_BF16, {"lagged_guiding": 1, "n_runs": 2, "loser_out": 1}),
    }


def _make(pkg, w, seed, prec, kw):
    X, y = (None, None) if w.kind == W.KIND_SPHERE else W.make_data(w)
    return pkg.Mgfwa.for_workload(w, seed, precision=prec, X=X, y=y, **kw)


@pytest.mark.parametrize("case", ["fp32", "bf16", "bf16_full", "fp8", "three_layer", "sphere", "two_runs", "refine",
                                  "loser_out", "lagged_bf16", "lagged_fp32", "lagged_two_runs_loser_out"])
def test_graph_replay_equals_kernel_by_kernel(pkg, case):
    spec = _specs(pkg)[case]
    states = []
    for timed in (True, False):
        with _make(pkg, *spec) as h:
            if timed:
                h.profile(True)   # kernel-by-kernel launches between events
            h.run()
            info = h.info()
            bests = [h.best(b) for b in range(h.cfg.n_runs)]
            states.append((bests, h.read(pkg.MGFWA_BUF_FW_F), h.read(pkg.MGFWA_BUF_FW_X), info.generations,
                           info.kernel_launches))
    (ba, fa, xa, ga, la), (bb, fb, xb, gb, lb) = states
    assert ga == gb and lb <= la
    assert np.array_equal(fa, fb) and np.array_equal(xa, xb)
    for (x1, f1, e1), (x2, f2, e2) in zip(ba, bb):
        assert np.array_equal(x1, x2) and f1 == f2 and e1 == e2
