"""Pins of the oracle's FP8 (E4M3) reference: the quantizer against torch's
float8_e4m3fn cast (a library routine) and the format's defining values, and
the FP8 objective against the pinned FP64 objective where quantization is
exact."""
import numpy as np
import pytest

import oracle
import workloads as W


def test_quantizer_matches_torch_cast():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8_e4m3fn")
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.uniform(-448, 448, 20000), rng.uniform(-0.05, 0.05, 20000),
                        rng.uniform(-2.0 ** -6, 2.0 ** -6, 20000)]).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(oracle.quantize_e4m3(v), ref)


def test_quantizer_defining_values():
    q = oracle.quantize_e4m3
    assert q(448.0) == 448.0 and q(500.0) == 448.0 and q(-1e9) == -448.0  # saturating
    assert q(2.0 ** -9) == 2.0 ** -9                                       # smallest subnormal
    assert q(2.0 ** -10) == 0.0                                            # tie to even (0)
    assert q(3 * 2.0 ** -10) == 2.0 ** -8                                  # tie to even (2 x 2^-9)
    assert q(1.0 + 2.0 ** -4) == 1.0 and q(1.0 + 3 * 2.0 ** -4) == 1.25    # ties at spacing 1/8
    assert q(1.0 + 2.0 ** -4 + 1e-9) == 1.125
    assert q(240.0) == 240.0 and q(15.0 / 16 * 2 ** -6 * 16) == 0.9375 * 2 ** -2
    # every E4M3 value is a fixed point
    vals = [s * (2.0 ** (e - 7)) * (1 + m / 8) for s in (1, -1) for e in range(1, 16) for m in range(8)]
    vals = [v for v in vals if abs(v) <= 448] + [s * m * 2.0 ** -9 for s in (1, -1) for m in range(8)]
    assert np.array_equal(q(np.array(vals)), np.array(vals))


def test_fp8_objective_equals_fp64_objective_when_exact():
    """With X, W1 and the scales on the E4M3 grid (powers of two), quantizing
    changes nothing and the FP8 objective is the pinned FP64 objective."""
    w = W.scaled(W.MLP_8_16_3, n_samples=40)
    rng = np.random.default_rng(5)
    grid = np.array([s * 2.0 ** e * (1 + m / 8) for s in (1, -1) for e in range(-3, 2) for m in range(8)])
    X = rng.choice(grid, size=(40, 8)).astype(np.float32)
    y = (np.arange(40) % 3).astype(np.int32)
    prob = oracle.Problem.for_workload(w, X, y)
    x = W.random_vectors(1, w.dim, -1, 1, 2)[0]
    x[:8 * 16] = rng.choice(grid, size=8 * 16)
    f64 = prob.fitness(x)
    f8 = oracle.fitness_fp8(prob, x, 4.0, 0.5)
    assert abs(f8 - f64) <= 1e-12 * abs(f64)
    # and a generic vector moves by the E4M3 rounding only
    x2 = W.random_vectors(1, w.dim, -1, 1, 9)[0]
    assert abs(oracle.fitness_fp8(prob, x2, 448.0 / 1.0, 448.0 / 1.0) - prob.fitness(x2)) < 0.2 * prob.fitness(x2)
