"""The allocation-free FP32 fitness entry point, mgfwa_evaluate_fp32_noalloc.

It serves callers that cannot call cudaMalloc: a process whose device memory
belongs to another framework's allocator, or a latency-critical loop where
cudaMalloc/cudaFree would synchronise the device.  The caller passes its own
device buffers; the kernels' scratch is a fixed array inside the library.

This test calls it through the C ABI twice in a row and compares each result
bit for bit with the handle-based FP32 path (mgfwa_evaluate), which runs the
same kernels in the same order.  The two calls differ in spark count and in
sample-tile count (the first covers more scratch entries than the second), so
a scratch entry that the second call failed to write would surface as a stale
value from the first.  It also checks that neither call allocates: the
device's free memory and torch's allocator counters are the same before and
after each call.  The device buffers come from torch, standing in for the
caller's own allocator.  This file runs last, so that a failure here leaves
every other test already run.
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


def _alloc_state(torch):
    free, _ = torch.cuda.mem_get_info()
    st = torch.cuda.memory_stats()
    return free, st.get("num_alloc_retries", 0), st.get("allocation.all.allocated", 0), \
        st.get("segment.all.allocated", 0)


def test_noalloc_matches_handle_path_on_two_calls(pkg):
    torch = pytest.importorskip("torch")
    # call 1: 1000 samples (8 sample tiles) x 24 sparks; call 2: 300 samples (3 tiles) x 17 sparks
    cases = [(1000, W.random_vectors(24, W.MLP_784_64_10.dim, -1.0, 1.0, seed=1)),
             (300, W.random_vectors(17, W.MLP_784_64_10.dim, -1.0, 1.0, seed=2))]
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream().cuda_stream
    prepared = []
    for n_samples, xs in cases:
        w = W.scaled(W.MLP_784_64_10, n_samples=n_samples, n_fireworks=2, sparks_per_firework=12,
                     guiding_per_firework=2)
        X, y = W.make_data(w)
        with pkg.Mgfwa.for_workload(w, 0, X=X, y=y) as run:
            ref = run.evaluate(xs, pkg.MGFWA_FP32)
        D = w.dim
        ld = (D + 3) // 4 * 4
        n = xs.shape[0]
        rows = torch.zeros((n, ld), dtype=torch.float32, device=dev)
        rows[:, :D] = torch.from_numpy(xs).to(dev)
        prepared.append((w, ref, torch.from_numpy(X).to(dev), torch.from_numpy(y).to(dev), rows, ld, n,
                         torch.full((n,), float("nan"), dtype=torch.float32, device=dev)))
    # set-up call: the first call on a device may load the library's device code there
    w, _, Xd, yd, rows, ld, n, out = prepared[0]
    pkg.mgfwa_evaluate_fp32_noalloc(w.widths, w.acts, w.n_samples, Xd.data_ptr(), yd.data_ptr(),
                                    rows.data_ptr(), ld, n, out.data_ptr(), stream)
    torch.cuda.synchronize()
    out.fill_(float("nan"))
    torch.cuda.synchronize()
    for w, ref, Xd, yd, rows, ld, n, out in prepared:
        before = _alloc_state(torch)
        pkg.mgfwa_evaluate_fp32_noalloc(w.widths, w.acts, w.n_samples, Xd.data_ptr(), yd.data_ptr(),
                                        rows.data_ptr(), ld, n, out.data_ptr(), stream)
        torch.cuda.synchronize()
        assert _alloc_state(torch) == before, "the call changed device or allocator memory"
        got = out.cpu().numpy()
        assert np.array_equal(got.view(np.uint32), ref.astype(np.float32).view(np.uint32)), \
            np.max(np.abs(got.astype(np.float64) - ref))


def test_noalloc_rejects_work_beyond_its_fixed_scratch(pkg):
    torch = pytest.importorskip("torch")
    w = W.MLP_784_64_10                       # 2048 samples = 16 sample tiles
    X, y = W.make_data(w)
    dev = torch.device("cuda", torch.cuda.current_device())
    Xd = torch.from_numpy(X).to(dev)
    yd = torch.from_numpy(y).to(dev)
    ld = (w.dim + 3) // 4 * 4
    rows = torch.zeros((4, ld), dtype=torch.float32, device=dev)
    out = torch.zeros(4, dtype=torch.float32, device=dev)
    with pytest.raises(pkg.MgfwaError) as e:
        # 16 tiles x 20,000 sparks > 262,144 partial sums: rejected before any launch
        pkg.mgfwa_evaluate_fp32_noalloc(w.widths, w.acts, w.n_samples, Xd.data_ptr(), yd.data_ptr(),
                                        rows.data_ptr(), ld, 20_000, out.data_ptr(), 0)
    assert e.value.status == pkg.MGFWA_EINVAL
    assert "scratch" in pkg.mgfwa_last_error()
    with pytest.raises(pkg.MgfwaError) as e:
        # more samples than the kernels' grid can carry
        pkg.mgfwa_evaluate_fp32_noalloc(w.widths, w.acts, 65535 * 128 + 1, Xd.data_ptr(), yd.data_ptr(),
                                        rows.data_ptr(), ld, 1, out.data_ptr(), 0)
    assert e.value.status == pkg.MGFWA_EINVAL
