"""Seeded synthetic workloads for MGFWA weight-space search.

This module is the one piece shared by the CUDA library's callers (tests,
bench) and by the CPU oracle's tests.  It holds problem definitions and
seeded input generators only: no step of the fireworks method lives here.

Each workload is the cross-entropy of a small multilayer perceptron whose
flattened parameters (torch ``nn.Linear`` order: W1[h1][d_in] row-major, b1,
W2[h2][h1], b2, ...) form the search vector, evaluated on one shared
synthetic labelled batch.  The paper (Sec. 4.1, Eq. 1) optimises the input of
a fixed network instead; the weight-space objective used here is the workload
this library is built for.  Labels are ``y_n = n mod C`` so that class sizes
are equal up to one sample.
"""
from __future__ import annotations

import dataclasses
from typing import Tuple

import numpy as np

ACT_TANH = 0
ACT_RELU = 1
ACT_GELU = 2

KIND_MLP_CE = 0
KIND_SPHERE = 1
KIND_NET_OUTPUT = 2   # the paper's testbed: minimise a fixed network's output over its input


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    kind: int                      # KIND_MLP_CE or KIND_SPHERE
    widths: Tuple[int, ...]        # layer widths d_in, h1, ..., C (MLP only)
    acts: Tuple[int, ...]          # activation per hidden layer (MLP only)
    n_samples: int                 # N (MLP only)
    dim: int                       # D
    lb: float
    ub: float
    n_fireworks: int               # mu
    sparks_per_firework: int       # lambda
    guiding_per_firework: int      # m
    sigma: float
    eval_budget: int
    data_recipe: str = "none"      # "mixture" or "prototypes" (MLP only)
    data_params: Tuple[float, ...] = ()
    data_seed: int = 0

    @property
    def sparks_per_generation(self) -> int:
        return self.n_fireworks * (self.sparks_per_firework + self.guiding_per_firework)

    def generations_in_budget(self) -> int:
        per = self.sparks_per_generation
        return max(0, (self.eval_budget - self.n_fireworks) // per)

    def flops_per_spark(self) -> float:
        """2 N sum(fan_in * fan_out): the dense multiply-adds of one fitness evaluation."""
        if self.kind == KIND_NET_OUTPUT:
            w = self.widths
            return 2.0 * sum(w[i] * w[i + 1] for i in range(len(w) - 1))
        if self.kind != KIND_MLP_CE:
            return 2.0 * self.dim
        w = self.widths
        return 2.0 * self.n_samples * sum(w[i] * w[i + 1] for i in range(len(w) - 1))


def mlp_param_count(widths) -> int:
    return int(sum(widths[i] * widths[i + 1] + widths[i + 1] for i in range(len(widths) - 1)))


def budget_for_generations(mu: int, lam: int, m: int, gens: int) -> int:
    return mu + gens * mu * (lam + m)


# ---------------------------------------------------------------------------
# The three MLP workloads and the sphere used for convergence checks.

MLP_8_16_3 = Workload(
    name="mlp8-16tanh-3_N512", kind=KIND_MLP_CE, widths=(8, 16, 3), acts=(ACT_TANH,),
    n_samples=512, dim=mlp_param_count((8, 16, 3)), lb=-5.0, ub=5.0,
    n_fireworks=5, sparks_per_firework=40, guiding_per_firework=4, sigma=0.2,
    eval_budget=20_000, data_recipe="mixture", data_params=(2.0, 1.0))

MLP_784_64_10 = Workload(
    name="mlp784-64relu-10_N2048", kind=KIND_MLP_CE, widths=(784, 64, 10), acts=(ACT_RELU,),
    n_samples=2048, dim=mlp_param_count((784, 64, 10)), lb=-1.0, ub=1.0,
    n_fireworks=5, sparks_per_firework=200, guiding_per_firework=8, sigma=0.2,
    eval_budget=budget_for_generations(5, 200, 8, 200), data_recipe="prototypes",
    data_params=(0.1,))

MLP_3072_128_64_10 = Workload(
    name="mlp3072-128relu-64relu-10_N4096", kind=KIND_MLP_CE, widths=(3072, 128, 64, 10),
    acts=(ACT_RELU, ACT_RELU), n_samples=4096, dim=mlp_param_count((3072, 128, 64, 10)),
    lb=-1.0, ub=1.0, n_fireworks=8, sparks_per_firework=256, guiding_per_firework=8,
    sigma=0.2, eval_budget=budget_for_generations(8, 256, 8, 100), data_recipe="mixture",
    data_params=(1.0, 0.5))

SPHERE_30 = Workload(
    name="sphere30", kind=KIND_SPHERE, widths=(), acts=(), n_samples=0, dim=30,
    lb=-5.0, ub=5.0, n_fireworks=5, sparks_per_firework=40, guiding_per_firework=4,
    sigma=0.2, eval_budget=100_000)

def table2_net(net_id: int, **over) -> Workload:
    """The paper's testbed network `net_id` of Table 2 (Sec. 4.1): minimise its scalar output over its input.
    Widths [input] + [hidden] * (layer_num + 1) + [1] (the reading under which nets 2-9 match the printed
    parameter counts), ReLU for odd ids and GELU for even ones, input box [-1, 1]^d (the paper states no
    bounds), the bench's population; weights from make_net."""
    rows = {1: (10, 16, 4), 2: (10, 32, 4), 3: (20, 16, 4), 4: (20, 32, 4), 5: (100, 64, 7), 6: (100, 128, 7),
            7: (200, 64, 7), 8: (200, 128, 7), 9: (1000, 256, 10), 10: (1000, 512, 10), 11: (2000, 256, 10),
            12: (2000, 512, 10)}
    d, h, layer_num = rows[net_id]
    widths = (d,) + (h,) * (layer_num + 1) + (1,)
    act = ACT_RELU if net_id % 2 else ACT_GELU
    kw = dict(name=f"net{net_id}_{d}-{h}x{layer_num + 1}-1", kind=KIND_NET_OUTPUT, widths=widths,
              acts=(act,) * (len(widths) - 2), n_samples=0, dim=d, lb=-1.0, ub=1.0, n_fireworks=5,
              sparks_per_firework=200, guiding_per_firework=8, sigma=0.2,
              eval_budget=budget_for_generations(5, 200, 8, 200), data_seed=net_id)
    kw.update(over)
    return Workload(**kw)


def make_net(w: Workload) -> np.ndarray:
    """The fixed parameters of a testbed network (nn.Linear order), each layer's weights and biases drawn
    U(-1/sqrt(fan_in), 1/sqrt(fan_in)) (torch's nn.Linear default; the paper does not state its init)."""
    rng = np.random.default_rng(1000 + w.data_seed)
    parts = []
    for i in range(len(w.widths) - 1):
        fi, fo = w.widths[i], w.widths[i + 1]
        bound = 1.0 / np.sqrt(fi)
        parts.append(rng.uniform(-bound, bound, size=fi * fo))
        parts.append(rng.uniform(-bound, bound, size=fo))
    return np.ascontiguousarray(np.concatenate(parts), dtype=np.float32)


ALL = {w.name: w for w in (MLP_8_16_3, MLP_784_64_10, MLP_3072_128_64_10, SPHERE_30)}


# ---------------------------------------------------------------------------
# Seeded data generators (FP64 draws, stored as FP32).

def _labels(n: int, c: int) -> np.ndarray:
    return (np.arange(n) % c).astype(np.int32)


def gaussian_mixture(n: int, d: int, c: int, center_sd: float, noise_sd: float,
                     seed: int) -> Tuple[np.ndarray, np.ndarray]:
    """Class centers ~ N(0, center_sd^2 I_d); samples = center + N(0, noise_sd^2 I_d)."""
    rng = np.random.default_rng(seed)
    centers = rng.normal(0.0, center_sd, size=(c, d))
    y = _labels(n, c)
    x = centers[y] + rng.normal(0.0, noise_sd, size=(n, d))
    return np.ascontiguousarray(x, dtype=np.float32), y


def clipped_prototypes(n: int, d: int, c: int, noise_sd: float,
                       seed: int) -> Tuple[np.ndarray, np.ndarray]:
    """Class prototypes ~ U(0,1)^d; samples = clip(prototype + N(0, noise_sd^2), 0, 1)."""
    rng = np.random.default_rng(seed)
    protos = rng.uniform(0.0, 1.0, size=(c, d))
    y = _labels(n, c)
    x = np.clip(protos[y] + rng.normal(0.0, noise_sd, size=(n, d)), 0.0, 1.0)
    return np.ascontiguousarray(x, dtype=np.float32), y


def make_data(w: Workload, n_samples: int | None = None) -> Tuple[np.ndarray, np.ndarray]:
    """The shared batch (X [N][d_in] FP32 row-major, y [N] int32) of a workload."""
    if w.kind != KIND_MLP_CE:
        return np.zeros((0, 0), np.float32), np.zeros((0,), np.int32)
    n = w.n_samples if n_samples is None else n_samples
    d, c = w.widths[0], w.widths[-1]
    if w.data_recipe == "prototypes":
        return clipped_prototypes(n, d, c, w.data_params[0], w.data_seed)
    if w.data_recipe == "mixture":
        return gaussian_mixture(n, d, c, w.data_params[0], w.data_params[1], w.data_seed)
    raise ValueError(f"unknown data recipe {w.data_recipe!r}")


def scaled(w: Workload, **changes) -> Workload:
    """A copy of a workload with some fields changed (dim follows the widths)."""
    fields = dataclasses.asdict(w)
    fields.update(changes)
    if fields["kind"] == KIND_MLP_CE:
        fields["dim"] = mlp_param_count(fields["widths"])
    fields["widths"] = tuple(fields["widths"])
    fields["acts"] = tuple(fields["acts"])
    fields["data_params"] = tuple(fields["data_params"])
    return Workload(**fields)


def random_vectors(n: int, dim: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """n seeded vectors uniform in [lo, hi]^dim (FP32) for fitness-only checks."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(n, dim)).astype(np.float32)



def mixed_batch(n: int, seed: int, generations: int = 10):
    """n MLP workloads of different shapes for batching many runs at once:
    D log-uniform in [195, 50,890] across the 8-16(tanh)-3 and d_in-64(ReLU)-10
    families (d_in a multiple of 16, 16..784; below D = 1,226 the 8-16-3 net),
    3..8 fireworks, 32..256 sparks per firework with 4 or 8 guiding sparks,
    each with its own Gaussian-mixture batch of 512..2048 samples, and a
    budget of `generations` generations."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        D = float(np.exp(rng.uniform(np.log(195.0), np.log(50890.0))))
        if D < 1226:
            widths, acts = (8, 16, 3), (ACT_TANH,)
        else:
            d_in = int(np.clip(round((D - 64 - 650) / 64 / 16) * 16, 16, 784))
            widths, acts = (d_in, 64, 10), (ACT_RELU,)
        m = int(rng.choice([4, 8]))
        lam = int(rng.choice([32, 64, 128, 256]))
        mu = int(rng.integers(3, 9))
        N = int(rng.integers(4, 17)) * 128
        w = Workload(name=f"mixed{k}", kind=KIND_MLP_CE, widths=widths, acts=acts, n_samples=N,
                     dim=mlp_param_count(widths), lb=-1.0, ub=1.0, n_fireworks=mu, sparks_per_firework=lam,
                     guiding_per_firework=m, sigma=0.2, eval_budget=budget_for_generations(mu, lam, m, generations),
                     data_recipe="mixture", data_params=(2.0, 1.0), data_seed=1000 + k)
        out.append(w)
    return out
