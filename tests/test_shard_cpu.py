"""The sharding seam of one run's fireworks, on CPU (no GPU): the host
reduction of the shards' best keys, the firework ranges, the configuration
checks, and two gloo ranks that each hold half of a run's fireworks and
reduce their keys through torch.distributed to the run's best.

A shard of a run holds a contiguous range of its fireworks and draws every
firework's sparks from the Philox units of its index in the whole run, so
the shards' fireworks are, bit for bit, the unsharded run's (checked on the
GPU in test_gpu_shard.py); here each rank takes its range of the oracle's
run of the whole problem and only the reduction to the run's best crosses
ranks."""
import math
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2501_03944_gb300 as p
    return p


def test_reduce_best_keys_orders_by_fitness_then_shard(pkg):
    K = pkg.mgfwa_best_key
    keys = [K(3.0, 0, 0, 0), K(1.5, 2, 0, 0), K(1.5, 1, 0, 0), K(float("nan"), 3, 0, 0)]
    out = pkg.mgfwa_reduce_best_keys(keys)
    assert (out.f, out.shard) == (1.5, 1)          # equal fitness: the first shard, as the first minimum
    out = pkg.mgfwa_reduce_best_keys([K(float("nan"), 0, 0, 0), K(math.inf, 1, 0, 0)])
    assert (out.f, out.shard) == (math.inf, 1)      # NaN ranks after +inf
    out = pkg.mgfwa_reduce_best_keys([K(float("nan"), 2, 0, 0), K(float("nan"), 1, 0, 0)])
    assert math.isnan(out.f) and out.shard == 1
    out = pkg.mgfwa_reduce_best_keys([K(-2.0, 4, 1, 0)])
    assert (out.f, out.shard, out.run) == (-2.0, 4, 1)
    with pytest.raises(pkg.MgfwaError):
        pkg.mgfwa_reduce_best_keys([])


def test_shard_ranges_partition_the_fireworks(pkg):
    for mu in (1, 2, 5, 8, 13):
        for n in range(1, mu + 1):
            ranges = [pkg.shard_range(mu, s, n) for s in range(n)]
            assert ranges[0][0] == 0 and ranges[-1][1] == mu
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            assert all(hi > lo for lo, hi in ranges)


def test_shard_configuration_is_validated_without_a_gpu(pkg):
    import workloads as W
    w = W.MLP_8_16_3
    X, y = W.make_data(w)
    for over in (dict(n_shards=6), dict(n_shards=2, shard_id=2), dict(n_shards=2, shard_id=-1),
                 dict(n_shards=1, shard_id=1), dict(n_shards=2, loser_out=1),
                 dict(n_shards=2, refine_every=1, refine_steps=1, refine_lr=0.1)):
        with pytest.raises(pkg.MgfwaError) as e:
            pkg.Mgfwa.for_workload(w, 0, X=X, y=y, **over)
        assert e.value.status == pkg.MGFWA_EINVAL, over


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    import paper_2501_03944_gb300 as pkg
    import workloads as W
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    w = W.scaled(W.MLP_8_16_3, n_samples=64, sparks_per_firework=8, guiding_per_firework=2)
    X, y = W.make_data(w)
    prob = oracle.Problem.for_workload(w, X, y)
    p = oracle.params_for(w)
    seed = 77
    # the whole run on the oracle, each rank keeping its own fireworks' fitness history
    fw_x, fw_a = oracle.init(p, seed)
    fw_f = prob.fitness_many(fw_x).astype(np.float32)
    hist = [fw_f.copy()]
    for gen in range(1, 4):
        out = oracle.generation(p, prob, seed, gen, fw_x, fw_a, fw_f)
        fw_x, fw_a, fw_f = out["fw_x"], out["fw_amp"], out["fw_f"]
        hist.append(fw_f.copy())
    hist = np.stack(hist)                        # [generations + 1][mu]
    lo, hi = pkg.shard_range(p.mu, rank, world)
    mine = pkg.mgfwa_best_key(float(hist[:, lo:hi].min()), rank, 0, 0)
    glob = pkg.allgather_reduce_best(mine)
    q.put((rank, float(glob.f), int(glob.shard), float(hist.min()),
           int(np.argmin(hist.min(axis=0))), lo, hi))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_runs_best(pkg):
    import oracle
    oracle.build()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    res.sort()
    ranges = {r[0]: (r[5], r[6]) for r in res}
    for rank, gf, gshard, best, best_fw, lo, hi in res:
        assert gf == best                          # every rank ends with the run's best fitness
        lo_w, hi_w = ranges[gshard]
        assert lo_w <= best_fw < hi_w              # held by the shard of the best firework
    assert len({(r[1], r[2]) for r in res}) == 1   # the same result on both ranks
