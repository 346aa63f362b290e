"""Sharding one run's fireworks (mgfwa_config.shard_id / n_shards) on the GPU.

Each shard handle holds a contiguous range of the run's fireworks and draws
every firework's sparks from the Philox units of its index in the whole run,
so after every generation its fireworks (positions, amplitudes, fitness)
equal the same fireworks of the unsharded run bit for bit (FP32, and BF16,
whose per-spark fitness does not depend on which sparks share a launch).
A shard runs exactly the generations the whole run's budget allows, and the
run's best is recovered from the shards' best keys through the reduce_best
hook (here the hook combines the keys of shard handles in the same
process; across processes it would gather them, see allgather_reduce_best).
"""
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
    (W.scaled(W.MLP_8_16_3, n_samples=300), 0, (2, 3)),
    (W.scaled(W.MLP_784_64_10, n_samples=300, n_fireworks=4, sparks_per_firework=16, guiding_per_firework=4), 1, (2,)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_shards_equal_the_unsharded_run_bitwise(pkg, case):
    w, prec, shard_counts = CASES[case]
    X, y = W.make_data(w)
    seed, gens = 31, 4
    bufs = (pkg.MGFWA_BUF_FW_X, pkg.MGFWA_BUF_FW_AMP, pkg.MGFWA_BUF_FW_F)
    for n in shard_counts:
        full = pkg.Mgfwa.for_workload(w, seed, precision=prec, X=X, y=y)
        shards = [pkg.Mgfwa.for_workload(w, seed, precision=prec, X=X, y=y, n_shards=n, shard_id=s)
                  for s in range(n)]
        ranges = [pkg.shard_range(w.n_fireworks, s, n) for s in range(n)]
        for g in range(gens + 1):
            if g:
                full.step(1)
                for sh in shards:
                    sh.step(1)
            want = [full.read(b) for b in bufs]
            for sh, (lo, hi) in zip(shards, ranges):
                assert sh.mu_local == hi - lo
                for b, v in zip(bufs, want):
                    got = sh.read(b)
                    assert np.array_equal(got.view(np.uint32), v[lo:hi].view(np.uint32)), (n, g, b)

        # the run's best from the shards' keys, through each shard's reduce_best hook
        def hook_for(me):
            return lambda key: pkg.mgfwa_reduce_best_keys([key] + [o.shard_key() for o in shards if o is not me])
        for sh in shards:
            sh.set_reduce_best(hook_for(sh))
        keys = [sh.global_best_key() for sh in shards]
        assert len({(k.f, k.shard) for k in keys}) == 1
        fx, ff, _ = full.best()
        assert keys[0].f == full.read(pkg.MGFWA_BUF_BEST_F)[0]
        sx, sf, _ = shards[keys[0].shard].best()
        assert np.array_equal(sx, fx) and sf == ff
        for sh in shards:
            sh.set_reduce_best(None)
        assert shards[-1].global_best_key().shard == n - 1     # without the hook: the shard's own key
        for sh in shards:
            sh.close()
        full.close()


def test_shards_run_the_whole_runs_generations(pkg):
    w = W.scaled(W.MLP_8_16_3, n_samples=128)
    X, y = W.make_data(w)
    P = w.n_fireworks * (w.sparks_per_firework + w.guiding_per_firework)
    w = W.scaled(w, eval_budget=w.n_fireworks + 3 * P + P // 2)     # three whole generations fit
    full = pkg.Mgfwa.for_workload(w, 5, X=X, y=y)
    full.run()
    shards = [pkg.Mgfwa.for_workload(w, 5, X=X, y=y, n_shards=3, shard_id=s) for s in range(3)]
    for sh in shards:
        sh.run()
        assert sh.info().generations == full.info().generations == 3
        lo, hi = pkg.shard_range(w.n_fireworks, sh.cfg.shard_id, 3)
        assert sh.info().evals == (hi - lo) * (1 + 3 * (w.sparks_per_firework + w.guiding_per_firework))
        assert np.array_equal(sh.read(pkg.MGFWA_BUF_FW_X), full.read(pkg.MGFWA_BUF_FW_X)[lo:hi])
        sh.close()
    full.close()
