"""Host-side checks of the serving runtime (include/mgfwa.h, Serving) that
need no GPU: argument validation, footprint-based rejection at submit, FIFO
bookkeeping, and that a request whose admission fails on the host (here:
no CUDA device, so the run's stream cannot be made) is reported FAILED with
its slot and memory given back."""
import pytest

import workloads as W


@pytest.fixture(scope="module")
def pkg():
    from paper_2501_03944_gb300 import build as b
    b.build()
    import paper_2501_03944_gb300 as p
    p.load_library()
    return p


def test_server_create_validates(pkg):
    for max_live, limit in ((0, 1 << 30), (2, 0), (-1, 5)):
        with pytest.raises(pkg.MgfwaError) as e:
            pkg.Server(max_live, limit)
        assert e.value.status == pkg.MGFWA_EINVAL


def test_footprint_grows_with_the_problem(pkg):
    w = W.MLP_8_16_3
    cfg, obj = pkg.workload_request(w, seed=1)
    f1 = pkg.mgfwa_footprint(cfg, obj)
    cfg4, obj4 = pkg.workload_request(w, seed=1, n_runs=4)
    f4 = pkg.mgfwa_footprint(cfg4, obj4)
    assert 0 < f1 < f4
    # sparks of 4 runs alone account for at least 3 more runs' spark rows
    assert f4 - f1 >= 3 * w.sparks_per_generation * w.dim * 4
    bad, bobj = pkg.workload_request(w, seed=1, sparks_per_firework=41)
    with pytest.raises(pkg.MgfwaError):
        pkg.mgfwa_footprint(bad, bobj)


def test_testbed_footprint_and_submit(pkg):
    """The testbed objective's arena holds the network's parameters and two hidden-activation buffers of
    [rows][widest hidden layer]; the server copies the parameters at submit."""
    w = W.table2_net(5)  # 100 -> 64 x 8 -> 1
    cfg, obj = pkg.workload_request(w, seed=1)
    fp = pkg.mgfwa_footprint(cfg, obj)
    params = W.mlp_param_count(w.widths)
    rows = w.sparks_per_generation
    assert fp >= 4 * (params + 2 * rows * 64 + rows * 128)
    with pkg.Server(1, 1 << 40) as s:
        rid = s.submit(cfg, obj)
        del obj
        import gc
        gc.collect()
        info = s.poll(rid)[0]
        assert info.state == pkg.MGFWA_REQ_QUEUED and info.footprint == fp


def test_lagged_guiding_footprint(pkg):
    """Lagged multi-guiding adds exactly its recorded vectors, [mu m][Dp] FP32 (256-byte aligned)."""
    w = W.MLP_8_16_3
    cfg, obj = pkg.workload_request(w, seed=1)
    lag, lobj = pkg.workload_request(w, seed=1, lagged_guiding=1)
    dp = (w.dim + 63) // 64 * 64
    gv = w.n_fireworks * w.guiding_per_firework * dp * 4
    assert pkg.mgfwa_footprint(lag, lobj) - pkg.mgfwa_footprint(cfg, obj) == (gv + 255) // 256 * 256


def test_submit_rejects_requests_larger_than_the_limit(pkg):
    cfg, obj = pkg.workload_request(W.MLP_8_16_3, seed=1)
    fp = pkg.mgfwa_footprint(cfg, obj)
    with pkg.Server(2, fp - 1) as s:
        with pytest.raises(pkg.MgfwaError) as e:
            s.submit(cfg, obj)
        assert e.value.status == pkg.MGFWA_EINVAL
        st = s.stats()
        assert st.submitted == 0 and st.queued == 0
    with pkg.Server(2, fp) as s:
        rid = s.submit(cfg, obj)
        info, _ = s.poll(rid)
        assert info.state == pkg.MGFWA_REQ_QUEUED and info.footprint == fp
        assert info.t_submit <= s.now()
        with pytest.raises(pkg.MgfwaError):
            s.poll(rid + 100)


def test_the_server_copies_the_objective_at_submit(pkg):
    """The caller's buffers may go away right after submit."""
    w = W.MLP_8_16_3
    with pkg.Server(1, 1 << 40) as s:
        cfg, obj = pkg.workload_request(w, seed=3)
        rid = s.submit(cfg, obj)
        del obj
        import gc
        gc.collect()
        assert s.poll(rid)[0].state == pkg.MGFWA_REQ_QUEUED


@pytest.mark.skipif(__import__("torch").cuda.is_available(), reason="checks the no-device failure path")
def test_admission_failure_on_the_host_is_reported(pkg):
    w = W.MLP_8_16_3
    with pkg.Server(2, 1 << 40) as s:
        ids = [s.submit(*pkg.workload_request(w, seed=k)) for k in range(3)]
        assert s.stats().queued == 3
        s.tick(1)
        st = s.stats()
        assert st.failed == 3 and st.live == 0 and st.queued == 0 and st.device_bytes_in_use == 0
        for rid in ids:
            info, _ = s.poll(rid)
            assert info.state == pkg.MGFWA_REQ_FAILED and info.status == pkg.MGFWA_ECUDA
