"""Serving: many optimisation requests sharing one GPU (include/mgfwa.h,
Serving).  The paper runs one optimisation per GPU; a server batches
independent requests by giving each its own handle and stream, so the only
claims to check are that sharing changes no result, that admission keeps
the live runs' device memory within the limit, and that requests arriving
while others run are admitted as slots free up (continuous batching)."""
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


def _mix(pkg):
    """Requests of four kinds and several budgets: (workload, seed, precision, data)."""
    small = W.MLP_8_16_3
    big = W.scaled(W.MLP_784_64_10, n_samples=300, n_fireworks=3, sparks_per_firework=20, guiding_per_firework=4)
    sph = W.SPHERE_30
    data_small, data_big = W.make_data(small), W.make_data(big)
    out = []
    for k in range(8):
        if k % 3 == 0:
            w = W.scaled(big, eval_budget=W.budget_for_generations(3, 20, 4, 3 + k))
            out.append((w, 100 + k, pkg.MGFWA_BF16, data_big))
        elif k % 3 == 1:
            w = W.scaled(small, eval_budget=W.budget_for_generations(5, 40, 4, 4 + 2 * k))
            out.append((w, 200 + k, pkg.MGFWA_FP32, data_small))
        else:
            w = W.scaled(sph, eval_budget=W.budget_for_generations(sph.n_fireworks, sph.sparks_per_firework,
                                                                   sph.guiding_per_firework, 5 + k))
            out.append((w, 300 + k, pkg.MGFWA_FP32, (None, None)))
    # the paper's testbed objective: the server copies the network's parameters at submit
    net = W.scaled(W.table2_net(5), sparks_per_firework=40, guiding_per_firework=4,
                   eval_budget=W.budget_for_generations(5, 40, 4, 6))
    out.append((net, 400, pkg.MGFWA_FP32, (None, None)))
    return out


def _alone(pkg, w, seed, prec, data):
    X, y = data
    with pkg.Mgfwa.for_workload(w, seed, precision=prec, X=X, y=y) as r:
        r.run()
        return r.best()


def _drain(pkg, s, ids, gens=1, limit=None, max_ticks=10_000):
    for _ in range(max_ticks):
        st = s.stats()
        if limit is not None:
            assert st.device_bytes_in_use <= limit
        if st.live == 0 and st.queued == 0:
            return
        s.tick(gens)
    raise AssertionError("server did not drain")


def test_footprint_is_the_handles_allocation(pkg):
    for w, seed, prec, (X, y) in _mix(pkg)[:3]:
        cfg, obj = pkg.workload_request(w, seed, prec, X=X, y=y)
        with pkg.Mgfwa.for_workload(w, seed, precision=prec, X=X, y=y) as r:
            assert pkg.mgfwa_footprint(cfg, obj) == r.info().device_bytes


@pytest.mark.parametrize("gens_per_tick", [1, 3])
def test_mixed_requests_equal_runs_made_alone(pkg, gens_per_tick):
    reqs = _mix(pkg)
    with pkg.Server(max_live=3, device_bytes_limit=1 << 34) as s:
        ids = [s.submit(*pkg.workload_request(w, seed, prec, X=d[0], y=d[1])) for w, seed, prec, d in reqs]
        _drain(pkg, s, ids, gens_per_tick)
        st = s.stats()
        assert st.completed == len(reqs) and st.failed == 0 and st.device_bytes_in_use == 0
        for rid, (w, seed, prec, d) in zip(ids, reqs):
            info, x = s.poll(rid, want_x=True)
            assert info.state == pkg.MGFWA_REQ_DONE
            ax, af, aev = _alone(pkg, w, seed, prec, d)
            assert np.array_equal(x, ax) and info.best_f == af and info.evals == aev, (w.name, seed)
            assert info.t_submit <= info.t_admit <= info.t_done
        assert st.sparks_evaluated == sum(
            w.generations_in_budget() * w.sparks_per_generation for w, _, _, _ in reqs)


def test_admission_respects_the_memory_limit(pkg):
    w, seed, prec, (X, y) = _mix(pkg)[0]
    cfg, obj = pkg.workload_request(w, seed, prec, X=X, y=y)
    fp = pkg.mgfwa_footprint(cfg, obj)
    limit = 2 * fp + fp // 2
    with pkg.Server(max_live=8, device_bytes_limit=limit) as s:
        ids = [s.submit(*pkg.workload_request(w, seed + k, prec, X=X, y=y)) for k in range(5)]
        s.tick(1)
        st = s.stats()
        assert st.live == 2 and st.queued == 3 and st.device_bytes_in_use == 2 * fp
        _drain(pkg, s, ids, 1, limit)
        for k, rid in enumerate(ids):
            info, x = s.poll(rid, want_x=True)
            ax, af, _ = _alone(pkg, w, seed + k, prec, (X, y))
            assert info.state == pkg.MGFWA_REQ_DONE and np.array_equal(x, ax) and info.best_f == af
        # FIFO: a later request is never admitted before an earlier one
        admits = [s.poll(rid)[0].t_admit for rid in ids]
        assert admits == sorted(admits)


def test_requests_arriving_while_others_run(pkg):
    reqs = _mix(pkg)
    with pkg.Server(max_live=2, device_bytes_limit=1 << 34) as s:
        ids = [s.submit(*pkg.workload_request(*reqs[0][:3], X=reqs[0][3][0], y=reqs[0][3][1]))]
        for w, seed, prec, d in reqs[1:]:
            s.tick(1)
            ids.append(s.submit(*pkg.workload_request(w, seed, prec, X=d[0], y=d[1])))
        _drain(pkg, s, ids)
        infos = [s.poll(rid)[0] for rid in ids]
        assert all(i.state == pkg.MGFWA_REQ_DONE for i in infos)
        # some request was admitted while an earlier one was still live
        assert any(infos[j].t_admit < infos[i].t_done for i in range(len(ids)) for j in range(i + 1, len(ids)))
        for rid, (w, seed, prec, d) in zip(ids, reqs):
            info, x = s.poll(rid, want_x=True)
            ax, af, _ = _alone(pkg, w, seed, prec, d)
            assert np.array_equal(x, ax) and info.best_f == af


def test_admission_never_exceeds_the_limit_over_a_long_trace(pkg):
    """120 requests of six footprints (sphere runs of several dimensions and populations, 8-16-3 nets)
    arriving a few per tick while others run: after every tick the live runs' device bytes stay within the
    limit and the live count within the slots, admission stays first-in first-out, and every request
    finishes with the evaluations its budget allows."""
    rng = np.random.default_rng(11)
    small = W.MLP_8_16_3
    data_small = W.make_data(small)
    kinds = []
    for dim, mu in ((30, 5), (200, 3), (1000, 4), (4000, 2)):
        kinds.append((W.scaled(W.SPHERE_30, dim=dim, n_fireworks=mu), (None, None)))
    kinds.append((W.scaled(small, n_fireworks=3), data_small))
    kinds.append((small, data_small))
    reqs = []
    for k in range(120):
        w, d = kinds[int(rng.integers(len(kinds)))]
        gens = int(rng.integers(2, 9))
        w = W.scaled(w, eval_budget=W.budget_for_generations(w.n_fireworks, w.sparks_per_firework,
                                                             w.guiding_per_firework, gens))
        reqs.append((w, 900 + k, d, gens))
    fps = [pkg.mgfwa_footprint(*pkg.workload_request(w, s, pkg.MGFWA_FP32, X=d[0], y=d[1])) for w, s, d, _ in reqs]
    limit = int(1.6 * max(fps))             # the largest fits, and the limit binds most ticks
    assert sum(sorted(fps)[-3:]) > limit
    max_live = 5
    with pkg.Server(max_live=max_live, device_bytes_limit=limit) as s:
        ids, nxt = [], 0
        for _ in range(20_000):
            for _ in range(int(rng.integers(0, 4))):
                if nxt < len(reqs):
                    w, seed, d, _ = reqs[nxt]
                    ids.append(s.submit(*pkg.workload_request(w, seed, pkg.MGFWA_FP32, X=d[0], y=d[1])))
                    nxt += 1
            st = s.stats()
            assert st.device_bytes_in_use <= limit and st.live <= max_live
            if nxt == len(reqs) and st.live == 0 and st.queued == 0:
                break
            s.tick(1)
            st = s.stats()
            assert st.device_bytes_in_use <= limit and st.live <= max_live
        infos = [s.poll(rid)[0] for rid in ids]
    assert len(infos) == len(reqs) and all(i.state == pkg.MGFWA_REQ_DONE for i in infos)
    admits = [i.t_admit for i in infos]
    assert admits == sorted(admits)
    for i, (w, _, _, gens) in zip(infos, reqs):
        assert i.evals == w.n_fireworks + gens * w.sparks_per_generation
