"""Pins of the oracle's testbed objective (the paper's Sec. 4.1, Eq. 1: the
output of a fixed network, minimised over its input), against closed forms
and torch's float64 layers (F.linear, ReLU, exact GELU) on the Table 2
shapes."""
import numpy as np
import pytest

import oracle
import workloads as W


def _torch_forward(w, params, x):
    torch = pytest.importorskip("torch")
    import torch.nn.functional as F
    a = torch.tensor(x, dtype=torch.float64)
    p = torch.tensor(params, dtype=torch.float64)
    off = 0
    for i in range(len(w.widths) - 1):
        fi, fo = w.widths[i], w.widths[i + 1]
        Wt = p[off:off + fi * fo].reshape(fo, fi)
        off += fi * fo
        b = p[off:off + fo]
        off += fo
        a = F.linear(a, Wt, b)
        if i + 2 < len(w.widths):
            a = F.relu(a) if w.acts[i] == W.ACT_RELU else F.gelu(a)
    return float(a[0])


@pytest.mark.parametrize("net_id", [1, 2, 3, 4, 5, 6, 7, 8])
def test_matches_torch_float64(net_id):
    w = W.table2_net(net_id)
    params = W.make_net(w)
    assert params.size == W.mlp_param_count(w.widths)
    prob = oracle.Problem.for_workload(w)
    rng = np.random.default_rng(net_id)
    for _ in range(3):
        x = rng.uniform(-1, 1, size=w.dim).astype(np.float32)
        ref = _torch_forward(w, params, x)
        assert abs(prob.fitness(x) - ref) <= 1e-12 * max(1.0, abs(ref))


def test_single_linear_layer_is_a_dot_product():
    w = W.Workload(name="lin", kind=W.KIND_NET_OUTPUT, widths=(7, 1), acts=(), n_samples=0, dim=7, lb=-1, ub=1,
                   n_fireworks=2, sparks_per_firework=8, guiding_per_firework=2, sigma=0.2, eval_budget=100)
    params = np.arange(1, 9, dtype=np.float32) / 8.0      # w = 1/8 .. 7/8, b = 1
    prob = oracle.Problem(oracle.NET_OUTPUT, 7, w.widths, (), params=params)
    x = np.array([1, -1, 0.5, 0, 2, -0.25, 1], np.float32)
    expect = float(np.dot(params[:7].astype(np.float64), x.astype(np.float64)) + params[7])
    assert prob.fitness(x) == expect


def test_dead_relu_layer_leaves_the_output_bias():
    widths = (5, 4, 3, 1)
    n = W.mlp_param_count(widths)
    params = np.random.default_rng(3).uniform(-1, 1, n).astype(np.float32)
    params[20:24] = -100.0                                 # b1: every first hidden unit negative for x in the box
    prob = oracle.Problem(oracle.NET_OUTPUT, 5, widths, (W.ACT_RELU, W.ACT_RELU), params=params)
    # layer 2 sees zeros: a2 = relu(b2); f = W3 relu(b2) + b3
    b2 = params[24 + 12:24 + 12 + 3].astype(np.float64)
    W3 = params[24 + 15:24 + 18].astype(np.float64)
    b3 = float(params[-1])
    expect = float(np.dot(W3, np.maximum(b2, 0.0)) + b3)
    for seed in range(3):
        x = np.random.default_rng(seed).uniform(-1, 1, 5).astype(np.float32)
        assert abs(prob.fitness(x) - expect) <= 1e-15


def test_gelu_fixed_points():
    # one hidden GELU unit with weight 1 and bias 0, output weight 1, bias 0: f(x) = gelu(x)
    params = np.array([1, 0, 1, 0], np.float32)
    prob = oracle.Problem(oracle.NET_OUTPUT, 1, (1, 1, 1), (W.ACT_GELU,), params=params)
    assert prob.fitness(np.array([0.0], np.float32)) == 0.0
    assert abs(prob.fitness(np.array([8.0], np.float32)) - 8.0) < 1e-12          # Phi(8) = 1 - 6e-16
    assert abs(prob.fitness(np.array([-8.0], np.float32))) < 1e-12
