"""The GPU testbed tests' rounding-error models, vectorised over rows for
speed, give what their one-row definitions give (the batched forms are the
ones the tests apply to every row)."""
import numpy as np
import pytest

import workloads as W
from test_gpu_net_output import _inputs, fp32_sigma, fp32_sigma_rows
from test_gpu_net_output_x3 import x3_sigma, x3_sigma_rows


@pytest.mark.parametrize("net_id", [1, 3, 6, 9])
def test_batched_models_equal_one_row_models(net_id):
    w = W.table2_net(net_id)
    params = W.make_net(w)
    xs = _inputs(w, 11, 40 + net_id)
    for rows, one in ((fp32_sigma_rows, fp32_sigma), (x3_sigma_rows, x3_sigma)):
        f, s = rows(w, params, xs, batch=4, n_threads=2)
        for i in (0, 1, 2, 5, 10):
            f1, s1 = one(w, params, xs[i])
            assert abs(f[i] - f1) <= 1e-12 * max(1.0, abs(f1)), (rows.__name__, i)
            assert abs(s[i] - s1) <= 1e-9 * s1 + 1e-300, (rows.__name__, i)
