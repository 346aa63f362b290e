"""MGFWA CPU oracle (FP64 fitness, exact-FP32 state) -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the bench's CPU-baseline
leg load this package.  It wraps the plain C oracle in this directory
(``philox.c``, ``objective.c``, ``mgfwa.c``) through ctypes; nothing here is
shared with the CUDA library.  ``build()`` compiles the C sources with gcc
(``-ffp-contract=off`` so that FP32 state arithmetic is never fused).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ("philox.c", "objective.c", "mgfwa.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

INIT, EXPLODE, MAP, GMAP = 0, 1, 2, 3
MLP_CE, SPHERE, NET_OUTPUT = 0, 1, 2
TANH, RELU = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so``; returns the path."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    hdr = os.path.join(_HERE, "oracle.h")
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr, __file__])
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int64), ("lb", ctypes.c_float), ("ub", ctypes.c_float),
                ("mu", ctypes.c_int32), ("lam", ctypes.c_int32), ("m", ctypes.c_int32),
                ("k", ctypes.c_int32), ("beta", ctypes.c_float), ("amp0", ctypes.c_float),
                ("c_a", ctypes.c_float), ("c_r", ctypes.c_float), ("refine_every", ctypes.c_int32),
                ("refine_steps", ctypes.c_int32), ("refine_lr", ctypes.c_float), ("loser_out", ctypes.c_int32),
                ("lagged_guiding", ctypes.c_int32)]


class Objective(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dim", ctypes.c_int64), ("n_layers", ctypes.c_int32),
                ("widths", ctypes.POINTER(ctypes.c_int32)), ("acts", ctypes.POINTER(ctypes.c_int32)),
                ("n_samples", ctypes.c_int64), ("X", ctypes.POINTER(ctypes.c_float)),
                ("y", ctypes.POINTER(ctypes.c_int32)), ("params", ctypes.POINTER(ctypes.c_float))]


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            f32p, i32p, u32p = (ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_uint32))
            f64p, i64p = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
            pp, op = ctypes.POINTER(Params), ctypes.POINTER(Objective)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32, ctypes.c_int64]
            L.orc_uniform.restype = ctypes.c_float
            L.orc_subset_size.argtypes = [ctypes.c_float, ctypes.c_int32]
            L.orc_subset_size.restype = ctypes.c_int32
            L.orc_fitness.argtypes = [op, f32p]
            L.orc_fitness.restype = ctypes.c_double
            L.orc_fitness_many.argtypes = [op, f32p, ctypes.c_int64, ctypes.c_int64, f64p, ctypes.c_int32]
            L.orc_init.argtypes = [pp, ctypes.c_uint64, f32p, f32p]
            L.orc_explode.argtypes = [pp, ctypes.c_uint64, ctypes.c_uint32, f32p, f32p, f32p]
            L.orc_rank.argtypes = [pp, f32p, i32p, i32p]
            L.orc_guide.argtypes = [pp, ctypes.c_uint64, ctypes.c_uint32, f32p, f32p, f32p, i32p, i32p, f32p]
            L.orc_select.argtypes = [pp, f32p, f32p, f32p, f32p, f32p, f32p, f32p, i32p]
            L.orc_guiding_vectors.argtypes = [pp, f32p, i32p, i32p, f32p]
            L.orc_guide_from.argtypes = [pp, ctypes.c_uint64, ctypes.c_uint32, f32p, f32p, f32p, f32p]
            L.orc_loser_out.argtypes = [pp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_float, f32p,
                                        f32p, f32p, f32p, i32p]
            L.orc_run.argtypes = [pp, op, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                  f32p, f64p, i64p, i32p, f32p]
            L.orc_run.restype = ctypes.c_int32
            L.orc_gradient.argtypes = [op, f32p, f64p]
            L.orc_gradient.restype = ctypes.c_double
            L.orc_refine.argtypes = [op, ctypes.c_int64, f32p, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, f32p]
            L.orc_refine.restype = ctypes.c_double
            L.orc_refine_cost.argtypes = [pp]
            L.orc_refine_cost.restype = ctypes.c_int64
            _lib = L
    return _lib


# ---------------------------------------------------------------------------
# Thin numpy-facing helpers.

def philox(ctr: Sequence[int], key: Sequence[int]) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return out


def uniform(seed: int, purpose: int, gen: int, unit: int, coord: int) -> float:
    return float(lib().orc_uniform(seed, purpose, gen, unit, coord))


def subset_size(sigma: float, g: int) -> int:
    return int(lib().orc_subset_size(sigma, g))


def make_params(dim, lb, ub, mu, lam, m, sigma=0.2, k=None, beta=1.0, amp0=None, c_a=1.2, c_r=0.9,
                refine_every=0, refine_steps=0, refine_lr=0.0, loser_out=0, lagged_guiding=0) -> Params:
    if k is None:
        k = subset_size(sigma, lam // m)
    if amp0 is None:
        amp0 = float(np.float32(ub) - np.float32(lb))
    return Params(dim, lb, ub, mu, lam, m, k, beta, amp0, c_a, c_r, refine_every, refine_steps, refine_lr,
                  loser_out, lagged_guiding)


def params_for(w, **over) -> Params:
    """Oracle parameters of a workloads.Workload (defaults: beta 1, A0 = ub - lb, 1.2 / 0.9)."""
    kw = dict(dim=w.dim, lb=w.lb, ub=w.ub, mu=w.n_fireworks, lam=w.sparks_per_firework,
              m=w.guiding_per_firework, sigma=w.sigma)
    kw.update(over)
    return make_params(**kw)


class Problem:
    """An objective plus the buffers it points into (kept alive here)."""

    def __init__(self, kind: int, dim: int, widths=(), acts=(), X=None, y=None, params=None):
        self.kind = kind
        self.widths = np.ascontiguousarray(widths, dtype=np.int32) if len(widths) else np.zeros(1, np.int32)
        self.acts = np.ascontiguousarray(acts, dtype=np.int32) if len(acts) else np.zeros(1, np.int32)
        self.X = np.ascontiguousarray(X if X is not None else np.zeros((1, 1)), dtype=np.float32)
        self.y = np.ascontiguousarray(y if y is not None else np.zeros(1), dtype=np.int32)
        n = 0 if X is None else self.X.shape[0]
        self.params = np.ascontiguousarray(params if params is not None else np.zeros(1), dtype=np.float32)
        self.obj = Objective(kind, dim, max(len(widths) - 1, 0), _p(self.widths, ctypes.c_int32),
                             _p(self.acts, ctypes.c_int32), n, _p(self.X, ctypes.c_float),
                             _p(self.y, ctypes.c_int32), _p(self.params, ctypes.c_float))

    @classmethod
    def for_workload(cls, w, X=None, y=None):
        if w.kind == SPHERE:
            return cls(SPHERE, w.dim)
        if w.kind == NET_OUTPUT:
            import workloads
            return cls(NET_OUTPUT, w.dim, w.widths, w.acts, params=workloads.make_net(w))
        if X is None:
            import workloads
            X, y = workloads.make_data(w)
        return cls(MLP_CE, w.dim, w.widths, w.acts, X, y)

    def fitness(self, x: np.ndarray) -> float:
        x = np.ascontiguousarray(x, dtype=np.float32)
        return float(lib().orc_fitness(ctypes.byref(self.obj), _p(x, ctypes.c_float)))

    def fitness_many(self, xs: np.ndarray, n_threads: int = 1) -> np.ndarray:
        xs = np.ascontiguousarray(xs, dtype=np.float32)
        out = np.zeros(xs.shape[0], dtype=np.float64)
        lib().orc_fitness_many(ctypes.byref(self.obj), _p(xs, ctypes.c_float), xs.shape[0], xs.shape[1],
                               _p(out, ctypes.c_double), n_threads)
        return out


def init(p: Params, seed: int):
    x = np.zeros((p.mu, p.dim), np.float32)
    a = np.zeros(p.mu, np.float32)
    lib().orc_init(ctypes.byref(p), seed, _p(x, ctypes.c_float), _p(a, ctypes.c_float))
    return x, a


def explode(p: Params, seed: int, gen: int, fw_x: np.ndarray, fw_amp: np.ndarray) -> np.ndarray:
    fw_x = np.ascontiguousarray(fw_x, np.float32)
    fw_amp = np.ascontiguousarray(fw_amp, np.float32)
    s = np.zeros((p.mu * p.lam, p.dim), np.float32)
    lib().orc_explode(ctypes.byref(p), seed, gen, _p(fw_x, ctypes.c_float), _p(fw_amp, ctypes.c_float),
                      _p(s, ctypes.c_float))
    return s


def rank(p: Params, fit_e: np.ndarray):
    f = np.ascontiguousarray(fit_e, np.float32)
    top = np.zeros((p.mu, p.m, p.k), np.int32)
    bot = np.zeros((p.mu, p.m, p.k), np.int32)
    lib().orc_rank(ctypes.byref(p), _p(f, ctypes.c_float), _p(top, ctypes.c_int32), _p(bot, ctypes.c_int32))
    return top, bot


def guide(p: Params, seed: int, gen: int, fw_x, fw_amp, sparks, top, bottom) -> np.ndarray:
    fw_x = np.ascontiguousarray(fw_x, np.float32)
    fw_amp = np.ascontiguousarray(fw_amp, np.float32)
    sparks = np.ascontiguousarray(sparks, np.float32)
    top = np.ascontiguousarray(top, np.int32)
    bottom = np.ascontiguousarray(bottom, np.int32)
    g = np.zeros((p.mu * p.m, p.dim), np.float32)
    lib().orc_guide(ctypes.byref(p), seed, gen, _p(fw_x, ctypes.c_float), _p(fw_amp, ctypes.c_float),
                    _p(sparks, ctypes.c_float), _p(top, ctypes.c_int32), _p(bottom, ctypes.c_int32),
                    _p(g, ctypes.c_float))
    return g


def guiding_vectors(p: Params, sparks, top, bottom) -> np.ndarray:
    """The guiding vectors GV [mu * m][D] alone (lagged multi-guiding)."""
    sparks = np.ascontiguousarray(sparks, np.float32)
    top = np.ascontiguousarray(top, np.int32)
    bottom = np.ascontiguousarray(bottom, np.int32)
    gv = np.zeros((p.mu * p.m, p.dim), np.float32)
    lib().orc_guiding_vectors(ctypes.byref(p), _p(sparks, ctypes.c_float), _p(top, ctypes.c_int32),
                              _p(bottom, ctypes.c_int32), _p(gv, ctypes.c_float))
    return gv


def guide_from(p: Params, seed: int, gen: int, fw_x, fw_amp, gv) -> np.ndarray:
    """Guiding sparks G = x + beta GV with the mapping, from given vectors (lagged multi-guiding)."""
    fw_x = np.ascontiguousarray(fw_x, np.float32)
    fw_amp = np.ascontiguousarray(fw_amp, np.float32)
    gv = np.ascontiguousarray(gv, np.float32)
    g = np.zeros((p.mu * p.m, p.dim), np.float32)
    lib().orc_guide_from(ctypes.byref(p), seed, gen, _p(fw_x, ctypes.c_float), _p(fw_amp, ctypes.c_float),
                         _p(gv, ctypes.c_float), _p(g, ctypes.c_float))
    return g


def select(p: Params, fit_e, fit_g, sparks, guides, fw_x, fw_amp, fw_f):
    """Returns updated copies (fw_x, fw_amp, fw_f, winner)."""
    fit_e = np.ascontiguousarray(fit_e, np.float32)
    fit_g = np.ascontiguousarray(fit_g, np.float32)
    sparks = np.ascontiguousarray(sparks, np.float32)
    guides = np.ascontiguousarray(guides, np.float32)
    fw_x = np.array(fw_x, np.float32, copy=True)
    fw_amp = np.array(fw_amp, np.float32, copy=True)
    fw_f = np.array(fw_f, np.float32, copy=True)
    win = np.zeros(p.mu, np.int32)
    lib().orc_select(ctypes.byref(p), _p(fit_e, ctypes.c_float), _p(fit_g, ctypes.c_float),
                     _p(sparks, ctypes.c_float), _p(guides, ctypes.c_float), _p(fw_x, ctypes.c_float),
                     _p(fw_amp, ctypes.c_float), _p(fw_f, ctypes.c_float), _p(win, ctypes.c_int32))
    return fw_x, fw_amp, fw_f, win


def loser_out(p: Params, seed: int, gen: int, g_rem: int, run_best: float, f_old, fw_x, fw_amp, fw_f):
    """The loser-out tournament after a selection: returns updated copies (fw_x, fw_amp, fw_f, loser)."""
    f_old = np.ascontiguousarray(f_old, np.float32)
    fw_x = np.array(fw_x, np.float32, copy=True)
    fw_amp = np.array(fw_amp, np.float32, copy=True)
    fw_f = np.array(fw_f, np.float32, copy=True)
    lo = np.zeros(p.mu, np.int32)
    lib().orc_loser_out(ctypes.byref(p), seed, gen, g_rem, float(run_best), _p(f_old, ctypes.c_float),
                        _p(fw_x, ctypes.c_float), _p(fw_amp, ctypes.c_float), _p(fw_f, ctypes.c_float),
                        _p(lo, ctypes.c_int32))
    return fw_x, fw_amp, fw_f, lo


def g_max(p: Params, budget: int) -> int:
    """Generations the budget allows at mu (lam + m) evaluations each, after the mu initial ones."""
    return max(0, (budget - p.mu) // (p.mu * (p.lam + p.m)))


def run(p: Params, prob: Problem, seed: int, budget: int, max_gens: int = 1 << 30,
        n_threads: int = 1, want_trace: bool = False):
    """A whole oracle run.  Returns dict(best_x, best_f, evals, gens, trace)."""
    best_x = np.zeros(p.dim, np.float32)
    best_f = ctypes.c_double(0.0)
    evals = ctypes.c_int64(0)
    gens = ctypes.c_int32(0)
    per = p.mu * (p.lam + p.m)
    cap = min(max_gens, max(0, (budget - p.mu) // per))
    trace = np.zeros(max(cap, 1), np.float32) if want_trace else None
    rc = lib().orc_run(ctypes.byref(p), ctypes.byref(prob.obj), seed, budget, min(max_gens, 1 << 30),
                       n_threads, _p(best_x, ctypes.c_float), ctypes.byref(best_f), ctypes.byref(evals),
                       ctypes.byref(gens), _p(trace, ctypes.c_float) if trace is not None else None)
    if rc != 0:
        raise ValueError("oracle run rejected its parameters")
    out = dict(best_x=best_x, best_f=best_f.value, evals=evals.value, gens=gens.value)
    if trace is not None:
        out["trace"] = trace[:gens.value]
    return out


def gradient(prob: Problem, x: np.ndarray):
    """(FP64 objective, FP64 gradient) at the FP32 vector x, by backpropagation."""
    x = np.ascontiguousarray(x, np.float32)
    g = np.zeros(x.shape[0], np.float64)
    f = lib().orc_gradient(ctypes.byref(prob.obj), _p(x, ctypes.c_float), _p(g, ctypes.c_double))
    return f, g


def refine(prob: Problem, x: np.ndarray, steps: int, lr: float, lb: float, ub: float):
    """(refined FP32 vector, its FP64 objective) after `steps` projected gradient steps."""
    x = np.ascontiguousarray(x, np.float32)
    out = np.zeros_like(x)
    f = lib().orc_refine(ctypes.byref(prob.obj), x.shape[0], _p(x, ctypes.c_float), steps, lr, lb, ub,
                         _p(out, ctypes.c_float))
    return out, f


def refine_cost(p: Params) -> int:
    return int(lib().orc_refine_cost(ctypes.byref(p)))


def generation(p: Params, prob: Problem, seed: int, gen: int, fw_x, fw_amp, fw_f, n_threads: int = 1,
               run_best=None, g_rem=None, gv_prev=None):
    """One oracle generation, returning every intermediate (for step-by-step parity).  With the loser-out
    tournament on (p.loser_out), run_best (the run's best-so-far before this generation) and g_rem (the
    generations the budget allows after this one) are needed.  With lagged multi-guiding
    (p.lagged_guiding), gv_prev is the previous generation's "gv" (None in generation 1)."""
    sparks = explode(p, seed, gen, fw_x, fw_amp)
    fit_e64 = prob.fitness_many(sparks, n_threads)
    fit_e = fit_e64.astype(np.float32)
    top, bot = rank(p, fit_e)
    if p.lagged_guiding and gv_prev is not None:
        guides = guide_from(p, seed, gen, fw_x, fw_amp, gv_prev)
    else:
        guides = guide(p, seed, gen, fw_x, fw_amp, sparks, top, bot)
    fit_g64 = prob.fitness_many(guides, n_threads)
    fit_g = fit_g64.astype(np.float32)
    nx, na, nf, win = select(p, fit_e, fit_g, sparks, guides, fw_x, fw_amp, fw_f)
    out = dict(sparks=sparks, fit_e64=fit_e64, fit_e=fit_e, top=top, bottom=bot, guides=guides,
               fit_g64=fit_g64, fit_g=fit_g, fw_x=nx, fw_amp=na, fw_f=nf, winner=win)
    if p.lagged_guiding:
        out["gv"] = guiding_vectors(p, sparks, top, bot)
    if p.loser_out:
        rb = np.float32(run_best)
        for f in nf:
            if _key(f) < _key(rb):
                rb = f
        out["run_best"] = rb
        out["fw_x"], out["fw_amp"], out["fw_f"], out["loser"] = loser_out(p, seed, gen, g_rem, rb,
                                                                          np.asarray(fw_f, np.float32), nx, na, nf)
    return out


def _key(f) -> float:
    return float("inf") if np.isnan(f) else float(f)


# ---------------------------------------------------------------------------
# FP8 (E4M3) operands: what the FP8 tensor-core path computes.

def quantize_e4m3(v) -> np.ndarray:
    """Round to the nearest value of the OCP FP8 E4M3 format, ties to even,
    saturating at +-448 (1 sign bit, 4 exponent bits with bias 7, 3 mantissa
    bits; normal values down to 2^-6, subnormals spaced 2^-9).  Exact: every
    step is a power-of-two scaling or np.rint of an FP64 value."""
    v = np.asarray(v, np.float64)
    a = np.abs(v)
    m, e = np.frexp(a)                     # a = m 2^e, m in [0.5, 1)
    spacing = np.where(a >= 2.0 ** -6, np.ldexp(1.0, e - 4), 2.0 ** -9)
    q = np.rint(a / spacing) * spacing
    q = np.minimum(q, 448.0)
    return np.copysign(q, v)


def fitness_fp8(prob: Problem, x: np.ndarray, inv_scale_x: float, inv_scale_w: float) -> float:
    """FP64 objective of the network the FP8 path evaluates: X and the first
    layer's weights each multiplied by their inverse scale in FP32 and rounded
    to E4M3, the first layer's products summed and multiplied back by
    1 / (inv_scale_x inv_scale_w), the rest of the MLP unchanged (the
    cross-entropy of orc_fitness)."""
    if prob.kind != MLP_CE:
        raise ValueError("FP8 objective is defined for MLPs")
    w = tuple(int(v) for v in prob.widths)
    X = np.asarray(prob.X, np.float32)
    y = np.asarray(prob.y)
    x = np.asarray(x, np.float32)
    fx, fw = np.float32(inv_scale_x), np.float32(inv_scale_w)
    Xq = quantize_e4m3(X * fx)
    d_in, h1 = w[0], w[1]
    W1q = quantize_e4m3(x[:d_in * h1].reshape(h1, d_in) * fw)
    scale = 1.0 / (float(fx) * float(fw))
    off = d_in * h1
    b1 = x[off:off + h1].astype(np.float64)
    off += h1
    a = (Xq @ W1q.T) * np.float64(np.float32(scale)) + b1
    acts = tuple(int(v) for v in prob.acts)
    for l in range(1, len(w) - 1):
        a = np.tanh(a) if acts[l - 1] == TANH else np.maximum(a, 0.0)
        fi, fo = w[l], w[l + 1]
        Wl = x[off:off + fi * fo].reshape(fo, fi).astype(np.float64)
        off += fi * fo
        bl = x[off:off + fo].astype(np.float64)
        off += fo
        a = a @ Wl.T + bl
    zmax = a.max(axis=1, keepdims=True)
    lse = zmax[:, 0] + np.log(np.exp(a - zmax).sum(axis=1))
    return float(np.mean(lse - a[np.arange(a.shape[0]), y]))
