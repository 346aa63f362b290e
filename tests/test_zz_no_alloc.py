"""The allocation-free FP32 fitness entry point, mgfwa_evaluate_fp32_noalloc.

It serves callers that cannot call cudaMalloc: a process whose device memory
belongs to another framework's allocator, or a latency-critical loop where
cudaMalloc/cudaFree would synchronise the device.  The caller passes its own
device buffers; the kernels' scratch is a fixed array inside the library.

This test calls it through the C ABI twice in a row, on different sparks,
and compares each result with the handle-based FP32 path (mgfwa_evaluate)
within the FP32 tolerance the other GPU tests use.  Its device buffers come
from torch, standing in for the caller's own allocator.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

FP32_RTOL = 1e-5
FP32_ATOL = 1e-5


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2501_03944_gb300 as p
    return p


def test_noalloc_matches_handle_path_on_two_calls(pkg):
    torch = pytest.importorskip("torch")
    w = W.scaled(W.MLP_784_64_10, n_samples=300, n_fireworks=2, sparks_per_firework=12, guiding_per_firework=2)
    X, y = W.make_data(w)
    D = w.dim
    batches = [W.random_vectors(24, D, -1.0, 1.0, seed=1), W.random_vectors(17, D, -1.0, 1.0, seed=2)]
    with pkg.Mgfwa.for_workload(w, 0, X=X, y=y) as run:
        refs = [run.evaluate(xs, pkg.MGFWA_FP32) for xs in batches]

    dev = torch.device("cuda", torch.cuda.current_device())
    Xd = torch.from_numpy(X).to(dev)
    yd = torch.from_numpy(y).to(dev)
    ld = (D + 3) // 4 * 4
    stream = torch.cuda.current_stream().cuda_stream
    for xs, ref in zip(batches, refs):
        n = xs.shape[0]
        rows = torch.zeros((n, ld), dtype=torch.float32, device=dev)
        rows[:, :D] = torch.from_numpy(xs).to(dev)
        out = torch.full((n,), float("nan"), dtype=torch.float32, device=dev)
        pkg.mgfwa_evaluate_fp32_noalloc(w.widths, w.acts, w.n_samples, Xd.data_ptr(), yd.data_ptr(),
                                        rows.data_ptr(), ld, n, out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref) <= FP32_RTOL * np.abs(ref) + FP32_ATOL), np.max(np.abs(got - ref))


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
