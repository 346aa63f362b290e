"""Python binding of the GPU-MGFWA C ABI (``include/mgfwa.h``).

Argument marshalling only: every step of a generation runs in the CUDA
kernels of ``libmgfwa.so`` (built in-tree by ``build.py``).  There is no CPU
or PyTorch fallback; importing the binding without the built library raises.

The C calls are exposed under their own names (``mgfwa_create``,
``mgfwa_step``, ...) with ctypes structures mirroring the header, plus a small
``Mgfwa`` class that owns a handle.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmgfwa.so")

MGFWA_OK, MGFWA_EINVAL, MGFWA_ENOMEM, MGFWA_ECUDA, MGFWA_ETIMEOUT, MGFWA_EBUDGET = range(6)
MGFWA_FP32, MGFWA_BF16, MGFWA_FP8, MGFWA_FP32X3 = 0, 1, 2, 3
MGFWA_OBJ_MLP_CE, MGFWA_OBJ_SPHERE, MGFWA_OBJ_NET_OUTPUT = 0, 1, 2
MGFWA_ACT_TANH, MGFWA_ACT_RELU, MGFWA_ACT_GELU = 0, 1, 2
(MGFWA_PHASE_EXPLODE, MGFWA_PHASE_EVAL_E, MGFWA_PHASE_RANK, MGFWA_PHASE_GUIDE, MGFWA_PHASE_EVAL_G,
 MGFWA_PHASE_RESCORE, MGFWA_PHASE_SELECT, MGFWA_PHASE_REFINE) = range(8)
(MGFWA_BUF_FW_X, MGFWA_BUF_FW_AMP, MGFWA_BUF_FW_F, MGFWA_BUF_SPARKS, MGFWA_BUF_GUIDES, MGFWA_BUF_FIT_E,
 MGFWA_BUF_FIT_G, MGFWA_BUF_TOP, MGFWA_BUF_BOTTOM, MGFWA_BUF_WINNER, MGFWA_BUF_BEST_X, MGFWA_BUF_BEST_F,
 MGFWA_BUF_REFINE_X, MGFWA_BUF_REFINE_F, MGFWA_BUF_REFINE_ELITE, MGFWA_BUF_LOSER, MGFWA_BUF_GV) = range(17)

STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EBUDGET"}

# Every symbol the headers declare (checked by the CPU test suite).
EXPORTS = ("mgfwa_config_init", "mgfwa_create", "mgfwa_step", "mgfwa_run", "mgfwa_best", "mgfwa_best_run",
           "mgfwa_evaluate",
           "mgfwa_get_info", "mgfwa_destroy", "mgfwa_last_error", "mgfwa_debug_phase", "mgfwa_debug_read",
           "mgfwa_debug_write", "mgfwa_debug_profile", "mgfwa_debug_kernel_times", "mgfwa_evaluate_fp32_noalloc",
           "mgfwa_debug_gradient", "mgfwa_debug_fp32_tc",
           "mgfwa_footprint", "mgfwa_server_create", "mgfwa_server_submit", "mgfwa_server_tick", "mgfwa_server_poll",
           "mgfwa_server_stats_get", "mgfwa_server_now", "mgfwa_server_destroy", "mgfwa_group_create",
           "mgfwa_group_step", "mgfwa_group_destroy", "mgfwa_checkpoint_size", "mgfwa_checkpoint_save",
           "mgfwa_checkpoint_load", "mgfwa_shard_key", "mgfwa_reduce_best_keys", "mgfwa_set_reduce_best",
           "mgfwa_global_best_key", "mgfwa_debug_wait_budget", "mgfwa_debug_pair_tile",
           "mgfwa_debug_set_pair_tile")
MGFWA_REQ_QUEUED, MGFWA_REQ_RUNNING, MGFWA_REQ_DONE, MGFWA_REQ_FAILED = range(4)
N_KERNEL_GROUPS = 9
KERNEL_GROUPS = ("explode", "fitness_explosion", "fitness_finish", "rank", "guide", "fitness_guiding", "select",
                 "elite_rescore", "refine")


class mgfwa_config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int64), ("lb", ctypes.c_float), ("ub", ctypes.c_float),
                ("n_fireworks", ctypes.c_int32), ("sparks_per_firework", ctypes.c_int32),
                ("guiding_per_firework", ctypes.c_int32), ("sigma", ctypes.c_float), ("boost", ctypes.c_float),
                ("amp_init", ctypes.c_float), ("c_amplify", ctypes.c_float), ("c_reduce", ctypes.c_float),
                ("eval_budget", ctypes.c_int64), ("seed", ctypes.c_uint64), ("precision", ctypes.c_int32),
                ("elite_rescore", ctypes.c_int32), ("n_runs", ctypes.c_int32), ("refine_every", ctypes.c_int32),
                ("refine_steps", ctypes.c_int32), ("refine_lr", ctypes.c_float), ("loser_out", ctypes.c_int32),
                ("lagged_guiding", ctypes.c_int32), ("shard_id", ctypes.c_int32), ("n_shards", ctypes.c_int32)]


class mgfwa_best_key(ctypes.Structure):
    _fields_ = [("f", ctypes.c_float), ("shard", ctypes.c_int32), ("run", ctypes.c_int32), ("pad", ctypes.c_int32)]


# int32_t (*)(void* ctx, mgfwa_best_key* key)
REDUCE_BEST_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(mgfwa_best_key))


class mgfwa_objective(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_layers", ctypes.c_int32),
                ("widths", ctypes.POINTER(ctypes.c_int32)), ("acts", ctypes.POINTER(ctypes.c_int32)),
                ("n_samples", ctypes.c_int64), ("X", ctypes.POINTER(ctypes.c_float)),
                ("y", ctypes.POINTER(ctypes.c_int32)), ("params", ctypes.POINTER(ctypes.c_float))]


class mgfwa_info(ctypes.Structure):
    _fields_ = [("evals", ctypes.c_int64), ("generations", ctypes.c_int32), ("k", ctypes.c_int32),
                ("dim_padded", ctypes.c_int64), ("sparks_per_gen", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("kernel_launches", ctypes.c_int64), ("n_runs", ctypes.c_int32),
                ("fp8_inv_scale_x", ctypes.c_float), ("fp8_inv_scale_w", ctypes.c_float)]


class mgfwa_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("evals", ctypes.c_int64),
                ("best_f", ctypes.c_double), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("footprint", ctypes.c_int64)]


class mgfwa_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("live", ctypes.c_int32), ("queued", ctypes.c_int32),
                ("device_bytes_in_use", ctypes.c_int64), ("sparks_evaluated", ctypes.c_int64)]


class MgfwaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def load_library(path: Optional[str] = None):
    """Load ``libmgfwa.so``; raises if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(path)
    vp, i32, i64, f32p = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_float)
    L.mgfwa_config_init.argtypes = [ctypes.POINTER(mgfwa_config)]
    L.mgfwa_create.argtypes = [ctypes.POINTER(mgfwa_config), ctypes.POINTER(mgfwa_objective), vp,
                               ctypes.POINTER(vp)]
    L.mgfwa_step.argtypes = [vp, i32]
    L.mgfwa_run.argtypes = [vp]
    L.mgfwa_best.argtypes = [vp, f32p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    L.mgfwa_best_run.argtypes = [vp, i32, f32p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    L.mgfwa_evaluate.argtypes = [vp, f32p, i64, i32, f32p]
    L.mgfwa_get_info.argtypes = [vp, ctypes.POINTER(mgfwa_info)]
    L.mgfwa_destroy.argtypes = [vp]
    L.mgfwa_destroy.restype = None
    L.mgfwa_last_error.argtypes = [vp]
    L.mgfwa_last_error.restype = ctypes.c_char_p
    L.mgfwa_debug_phase.argtypes = [vp, i32]
    L.mgfwa_debug_read.argtypes = [vp, i32, vp, i64]
    L.mgfwa_debug_write.argtypes = [vp, i32, vp, i64]
    L.mgfwa_debug_profile.argtypes = [vp, i32]
    L.mgfwa_debug_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    L.mgfwa_debug_gradient.argtypes = [vp, f32p, i32, f32p, f32p]
    L.mgfwa_debug_fp32_tc.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    i32p = ctypes.POINTER(ctypes.c_int32)
    L.mgfwa_evaluate_fp32_noalloc.argtypes = [i32, i32p, i32p, i64, vp, vp, vp, i64, i32, vp, vp]
    L.mgfwa_shard_key.argtypes = [vp, i32, ctypes.POINTER(mgfwa_best_key)]
    L.mgfwa_debug_wait_budget.argtypes = [vp, ctypes.c_uint64]
    L.mgfwa_debug_pair_tile.argtypes = [vp, i32p, i32p, i32p, i32p]
    L.mgfwa_debug_set_pair_tile.argtypes = [vp, i32, i32, i32]
    L.mgfwa_reduce_best_keys.argtypes = [ctypes.POINTER(mgfwa_best_key), i32, ctypes.POINTER(mgfwa_best_key)]
    L.mgfwa_set_reduce_best.argtypes = [vp, REDUCE_BEST_FN, vp]
    L.mgfwa_global_best_key.argtypes = [vp, i32, ctypes.POINTER(mgfwa_best_key)]
    L.mgfwa_footprint.argtypes = [ctypes.POINTER(mgfwa_config), ctypes.POINTER(mgfwa_objective),
                                  ctypes.POINTER(ctypes.c_int64)]
    L.mgfwa_server_create.argtypes = [i32, i64, ctypes.POINTER(vp)]
    L.mgfwa_server_submit.argtypes = [vp, ctypes.POINTER(mgfwa_config), ctypes.POINTER(mgfwa_objective),
                                      ctypes.POINTER(ctypes.c_int64)]
    L.mgfwa_server_tick.argtypes = [vp, i32]
    L.mgfwa_server_poll.argtypes = [vp, i64, ctypes.POINTER(mgfwa_request_info), f32p]
    L.mgfwa_server_stats_get.argtypes = [vp, ctypes.POINTER(mgfwa_server_stats)]
    L.mgfwa_server_now.argtypes = [vp]
    L.mgfwa_server_now.restype = ctypes.c_double
    L.mgfwa_server_destroy.argtypes = [vp]
    L.mgfwa_server_destroy.restype = None
    L.mgfwa_group_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp)]
    L.mgfwa_group_step.argtypes = [vp, i32]
    L.mgfwa_group_destroy.argtypes = [vp]
    L.mgfwa_checkpoint_size.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    L.mgfwa_checkpoint_save.argtypes = [vp, vp, i64]
    L.mgfwa_checkpoint_load.argtypes = [vp, vp, i64]
    L.mgfwa_group_destroy.restype = None
    for name in EXPORTS:
        if name not in ("mgfwa_destroy", "mgfwa_last_error", "mgfwa_server_now", "mgfwa_server_destroy",
                        "mgfwa_group_destroy"):
            getattr(L, name).restype = ctypes.c_int
    if path == LIB_PATH:
        _lib = L
    return L


def _f32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if a is not None else None


# ---------------------------------------------------------------------------
# The C calls under their own names.

def mgfwa_config_init() -> mgfwa_config:
    cfg = mgfwa_config()
    load_library().mgfwa_config_init(ctypes.byref(cfg))
    return cfg


def mgfwa_last_error(handle=None) -> str:
    return load_library().mgfwa_last_error(handle).decode()


def _check(st: int, handle=None):
    if st != MGFWA_OK:
        raise MgfwaError(st, mgfwa_last_error(handle))


class _ObjectiveBuffers:
    def __init__(self, kind, widths=(), acts=(), X=None, y=None, params=None):
        self.widths = np.ascontiguousarray(widths if len(widths) else [0], dtype=np.int32)
        self.acts = np.ascontiguousarray(acts if len(acts) else [0], dtype=np.int32)
        self.X = np.ascontiguousarray(X if X is not None else np.zeros((1, 1)), dtype=np.float32)
        self.y = np.ascontiguousarray(y if y is not None else np.zeros(1), dtype=np.int32)
        self.obj = mgfwa_objective(kind, max(len(widths) - 1, 0),
                                   self.widths.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   self.acts.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   0 if X is None else self.X.shape[0], _f32p(self.X),
                                   self.y.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        # the testbed network's fixed parameters (kept alive with the struct)
        self.params = None if params is None else np.ascontiguousarray(params, dtype=np.float32).ravel()
        if self.params is not None:
            self.obj.params = _f32p(self.params)


def mgfwa_create(cfg: mgfwa_config, objective: mgfwa_objective, stream: int = 0) -> int:
    h = ctypes.c_void_p()
    st = load_library().mgfwa_create(ctypes.byref(cfg), ctypes.byref(objective),
                                     ctypes.c_void_p(stream or None), ctypes.byref(h))
    _check(st)
    return h.value


def mgfwa_step(handle: int, n_generations: int) -> int:
    return load_library().mgfwa_step(handle, n_generations)


def mgfwa_run(handle: int) -> int:
    return load_library().mgfwa_run(handle)


def mgfwa_best(handle: int, dim: int):
    x = np.zeros(dim, np.float32)
    f = ctypes.c_double()
    ev = ctypes.c_int64()
    _check(load_library().mgfwa_best(handle, _f32p(x), ctypes.byref(f), ctypes.byref(ev)), handle)
    return x, f.value, ev.value


def mgfwa_best_run(handle: int, run: int, dim: int):
    x = np.zeros(dim, np.float32)
    f = ctypes.c_double()
    ev = ctypes.c_int64()
    _check(load_library().mgfwa_best_run(handle, run, _f32p(x), ctypes.byref(f), ctypes.byref(ev)), handle)
    return x, f.value, ev.value


def mgfwa_evaluate(handle: int, xs: np.ndarray, precision: int) -> np.ndarray:
    xs = np.ascontiguousarray(xs, np.float32)
    out = np.zeros(xs.shape[0], np.float32)
    _check(load_library().mgfwa_evaluate(handle, _f32p(xs), xs.shape[0], precision, _f32p(out)), handle)
    return out


def mgfwa_get_info(handle: int) -> mgfwa_info:
    info = mgfwa_info()
    _check(load_library().mgfwa_get_info(handle, ctypes.byref(info)), handle)
    return info


def mgfwa_destroy(handle: int) -> None:
    load_library().mgfwa_destroy(handle)


def mgfwa_evaluate_fp32_noalloc(widths, acts, n_samples: int, X_dev: int, y_dev: int, rows_dev: int, ld: int,
                                count: int, fitness_dev: int, stream: int = 0) -> None:
    """FP32 fitness of caller-owned device buffers (integer device addresses); allocates nothing."""
    w = np.ascontiguousarray(widths, dtype=np.int32)
    a = np.ascontiguousarray(acts if len(acts) else [0], dtype=np.int32)
    i32p = ctypes.POINTER(ctypes.c_int32)
    st = load_library().mgfwa_evaluate_fp32_noalloc(len(widths) - 1, w.ctypes.data_as(i32p), a.ctypes.data_as(i32p),
                                                    n_samples, X_dev, y_dev, rows_dev, ld, count, fitness_dev,
                                                    ctypes.c_void_p(stream or None))
    _check(st)


def mgfwa_reduce_best_keys(keys) -> mgfwa_best_key:
    """The run's best of the shards' keys (host reduction in the library): smallest f, NaN last, then shard."""
    arr = (mgfwa_best_key * len(keys))(*keys)
    out = mgfwa_best_key()
    _check(load_library().mgfwa_reduce_best_keys(arr, len(keys), ctypes.byref(out)))
    return out


def shard_range(n_fireworks: int, shard_id: int, n_shards: int):
    """Fireworks [lo, hi) of the run that shard `shard_id` of `n_shards` holds."""
    n = max(n_shards, 1)
    return shard_id * n_fireworks // n, (shard_id + 1) * n_fireworks // n


def mgfwa_debug_phase(handle: int, phase: int) -> int:
    return load_library().mgfwa_debug_phase(handle, phase)


def mgfwa_debug_read(handle: int, buf: int, out: np.ndarray) -> np.ndarray:
    out = np.ascontiguousarray(out)
    _check(load_library().mgfwa_debug_read(handle, buf, out.ctypes.data, out.nbytes), handle)
    return out


def mgfwa_debug_write(handle: int, buf: int, src: np.ndarray) -> None:
    src = np.ascontiguousarray(src)
    _check(load_library().mgfwa_debug_write(handle, buf, src.ctypes.data, src.nbytes), handle)


def mgfwa_debug_fp32_tc(handle: int) -> tuple:
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(load_library().mgfwa_debug_fp32_tc(handle, ctypes.byref(a), ctypes.byref(b)), handle)
    return a.value, b.value


# ---------------------------------------------------------------------------
# Convenience owner of one handle.

class Mgfwa:
    """One MGFWA run on the GPU, configured from plain values or a workloads.Workload."""

    def __init__(self, *, dim, lb, ub, n_fireworks, sparks_per_firework, guiding_per_firework, eval_budget,
                 seed, sigma=0.2, boost=1.0, amp_init=0.0, c_amplify=1.2, c_reduce=0.9, precision=MGFWA_FP32,
                 kind=MGFWA_OBJ_MLP_CE, widths=(), acts=(), X=None, y=None, stream: int = 0, n_runs: int = 1,
                 elite_rescore: int = 2, refine_every: int = 0, refine_steps: int = 0, refine_lr: float = 0.0,
                 loser_out: int = 0, params=None, lagged_guiding: int = 0, shard_id: int = 0, n_shards: int = 1):
        cfg = mgfwa_config_init()
        cfg.dim, cfg.lb, cfg.ub = dim, lb, ub
        cfg.n_fireworks, cfg.sparks_per_firework, cfg.guiding_per_firework = (
            n_fireworks, sparks_per_firework, guiding_per_firework)
        cfg.sigma, cfg.boost, cfg.amp_init, cfg.c_amplify, cfg.c_reduce = sigma, boost, amp_init, c_amplify, c_reduce
        cfg.eval_budget, cfg.seed, cfg.precision = eval_budget, seed, precision
        cfg.n_runs = n_runs
        cfg.elite_rescore = elite_rescore
        cfg.refine_every, cfg.refine_steps, cfg.refine_lr = refine_every, refine_steps, refine_lr
        cfg.loser_out = loser_out
        cfg.lagged_guiding = lagged_guiding
        cfg.shard_id, cfg.n_shards = shard_id, n_shards
        self.cfg = cfg
        lo, hi = shard_range(n_fireworks, shard_id, n_shards)
        self.mu_local = hi - lo          # fireworks this handle holds
        self._hook = None
        self._obj = _ObjectiveBuffers(kind, widths, acts, X, y, params)
        self.dim = dim
        self.handle = mgfwa_create(cfg, self._obj.obj, stream)
        info = mgfwa_get_info(self.handle)
        self.k = info.k
        self.sparks_per_gen = info.sparks_per_gen

    @classmethod
    def for_workload(cls, w, seed: int, precision: int = MGFWA_FP32, X=None, y=None, **over):
        kw = dict(dim=w.dim, lb=w.lb, ub=w.ub, n_fireworks=w.n_fireworks, sparks_per_firework=w.sparks_per_firework,
                  guiding_per_firework=w.guiding_per_firework, eval_budget=w.eval_budget, seed=seed,
                  sigma=w.sigma, precision=precision, kind=w.kind)
        if w.kind == MGFWA_OBJ_MLP_CE:
            if X is None:
                import workloads
                X, y = workloads.make_data(w)
            kw.update(widths=w.widths, acts=w.acts, X=X, y=y)
        elif w.kind == MGFWA_OBJ_NET_OUTPUT:
            import workloads
            kw.update(widths=w.widths, acts=w.acts, params=workloads.make_net(w))
        kw.update(over)
        return cls(**kw)

    def step(self, n: int = 1) -> int:
        st = mgfwa_step(self.handle, n)
        if st not in (MGFWA_OK, MGFWA_EBUDGET):
            _check(st, self.handle)
        return st

    def run(self) -> None:
        _check(mgfwa_run(self.handle), self.handle)

    def best(self, run: Optional[int] = None):
        if run is None:
            return mgfwa_best(self.handle, self.dim)
        return mgfwa_best_run(self.handle, run, self.dim)

    def evaluate(self, xs, precision: Optional[int] = None) -> np.ndarray:
        return mgfwa_evaluate(self.handle, xs, self.cfg.precision if precision is None else precision)

    def info(self) -> mgfwa_info:
        return mgfwa_get_info(self.handle)

    def phase(self, ph: int) -> None:
        _check(mgfwa_debug_phase(self.handle, ph), self.handle)

    def wait_budget(self, ticks: int) -> None:
        """Budget (SM clock ticks) of the tensor-core kernels' bounded waits; 0 restores the default."""
        _check(load_library().mgfwa_debug_wait_budget(self.handle, ticks), self.handle)

    def pair_tile(self) -> tuple:
        """(sparks per tile, stages, tuned, K-tail MMAs) of the CTA-pair fitness kernel; all -1 off that kernel."""
        v = [ctypes.c_int32() for _ in range(4)]
        _check(load_library().mgfwa_debug_pair_tile(self.handle, *[ctypes.byref(x) for x in v]), self.handle)
        return tuple(x.value for x in v)

    def set_pair_tile(self, sparks_per_tile: int, stages: int, k_tail: int = -1) -> None:
        """Run the following generations with this tile of the CTA-pair fitness kernel (k_tail: 1 the partial
        last K atom through the K-tail buffers, 0 as a pipeline stage, -1 the buffers where they fit)."""
        _check(load_library().mgfwa_debug_set_pair_tile(self.handle, sparks_per_tile, stages, k_tail), self.handle)

    def shard_key(self, run: int = 0) -> mgfwa_best_key:
        key = mgfwa_best_key()
        _check(load_library().mgfwa_shard_key(self.handle, run, ctypes.byref(key)), self.handle)
        return key

    def set_reduce_best(self, fn) -> None:
        """Register fn(key) -> key (the combination of this shard's key with the other shards', e.g. over
        torch.distributed) as the handle's reduce_best hook; None removes it."""
        if fn is None:
            self._hook = None
            _check(load_library().mgfwa_set_reduce_best(self.handle, REDUCE_BEST_FN(), None), self.handle)
            return

        def hook(ctx, key_p):
            try:
                out = fn(mgfwa_best_key(key_p[0].f, key_p[0].shard, key_p[0].run, 0))
                key_p[0] = out
                return 0
            except Exception:  # noqa: BLE001 - a failing hook is reported through the status
                return 1
        self._hook = REDUCE_BEST_FN(hook)  # kept alive with the handle
        _check(load_library().mgfwa_set_reduce_best(self.handle, self._hook, None), self.handle)

    def global_best_key(self, run: int = 0) -> mgfwa_best_key:
        key = mgfwa_best_key()
        _check(load_library().mgfwa_global_best_key(self.handle, run, ctypes.byref(key)), self.handle)
        return key

    def read(self, buf: int) -> np.ndarray:
        B = self.cfg.n_runs
        mu, lam, m, D, k = (B * self.mu_local, self.cfg.sparks_per_firework, self.cfg.guiding_per_firework,
                            self.dim, self.k)
        shapes = {MGFWA_BUF_FW_X: ((mu, D), np.float32), MGFWA_BUF_FW_AMP: ((mu,), np.float32),
                  MGFWA_BUF_FW_F: ((mu,), np.float32), MGFWA_BUF_SPARKS: ((mu * lam, D), np.float32),
                  MGFWA_BUF_GUIDES: ((mu * m, D), np.float32), MGFWA_BUF_FIT_E: ((mu * lam,), np.float32),
                  MGFWA_BUF_FIT_G: ((mu * m,), np.float32), MGFWA_BUF_TOP: ((mu, m, k), np.int32),
                  MGFWA_BUF_BOTTOM: ((mu, m, k), np.int32), MGFWA_BUF_WINNER: ((mu,), np.int32),
                  MGFWA_BUF_BEST_X: ((B, D) if B > 1 else (D,), np.float32), MGFWA_BUF_BEST_F: ((B,), np.float32),
                  MGFWA_BUF_REFINE_X: ((B, D), np.float32), MGFWA_BUF_REFINE_F: ((B,), np.float32),
                  MGFWA_BUF_REFINE_ELITE: ((B,), np.int32), MGFWA_BUF_LOSER: ((mu,), np.int32),
                  MGFWA_BUF_GV: ((mu * m, D), np.float32)}
        shape, dt = shapes[buf]
        return mgfwa_debug_read(self.handle, buf, np.zeros(shape, dt))

    def write(self, buf: int, arr: np.ndarray) -> None:
        mgfwa_debug_write(self.handle, buf, arr)

    def checkpoint(self) -> bytes:
        """The run's state (see include/mgfwa.h, Checkpoint / resume)."""
        L = load_library()
        n = ctypes.c_int64()
        _check(L.mgfwa_checkpoint_size(self.handle, ctypes.byref(n)), self.handle)
        buf = ctypes.create_string_buffer(n.value)
        _check(L.mgfwa_checkpoint_save(self.handle, buf, n.value), self.handle)
        return buf.raw

    def restore(self, data: bytes) -> None:
        buf = ctypes.create_string_buffer(data, len(data))
        _check(load_library().mgfwa_checkpoint_load(self.handle, buf, len(data)), self.handle)

    def gradient(self, xs):
        """(FP32 objective [count], FP32 gradient [count][D]) of host vectors, by the refinement's kernels."""
        xs = np.ascontiguousarray(np.atleast_2d(xs), np.float32)
        g = np.zeros_like(xs)
        f = np.zeros(xs.shape[0], np.float32)
        _check(load_library().mgfwa_debug_gradient(self.handle, _f32p(xs), xs.shape[0], _f32p(g), _f32p(f)),
               self.handle)
        return f, g

    def fp32_tensor_cores(self) -> tuple:
        """(re-score, refinement): 1 where the FP32-accurate tensor-core first layer serves it, 0 where the
        CUDA-core products do, -1 where the handle has no such phase."""
        return mgfwa_debug_fp32_tc(self.handle)

    def profile(self, enable: bool = True) -> None:
        _check(load_library().mgfwa_debug_profile(self.handle, int(enable)), self.handle)

    def kernel_times(self) -> dict:
        """{group: (total ms, launches)} since the last profile(True)."""
        ms = (ctypes.c_double * N_KERNEL_GROUPS)()
        n = (ctypes.c_int64 * N_KERNEL_GROUPS)()
        _check(load_library().mgfwa_debug_kernel_times(self.handle, ms, n), self.handle)
        return {g: (ms[i], n[i]) for i, g in enumerate(KERNEL_GROUPS)}

    def close(self) -> None:
        if getattr(self, "handle", None):
            mgfwa_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Serving (continuous batching of optimisation requests on one GPU).

def make_config(*, dim, lb, ub, n_fireworks, sparks_per_firework, guiding_per_firework, eval_budget, seed,
                sigma=0.2, boost=1.0, amp_init=0.0, c_amplify=1.2, c_reduce=0.9, precision=MGFWA_FP32, n_runs=1,
                elite_rescore=2, refine_every=0, refine_steps=0, refine_lr=0.0, loser_out=0,
                lagged_guiding=0) -> mgfwa_config:
    cfg = mgfwa_config_init()
    cfg.dim, cfg.lb, cfg.ub = dim, lb, ub
    cfg.n_fireworks, cfg.sparks_per_firework, cfg.guiding_per_firework = (
        n_fireworks, sparks_per_firework, guiding_per_firework)
    cfg.sigma, cfg.boost, cfg.amp_init, cfg.c_amplify, cfg.c_reduce = sigma, boost, amp_init, c_amplify, c_reduce
    cfg.eval_budget, cfg.seed, cfg.precision, cfg.n_runs, cfg.elite_rescore = (
        eval_budget, seed, precision, n_runs, elite_rescore)
    cfg.refine_every, cfg.refine_steps, cfg.refine_lr = refine_every, refine_steps, refine_lr
    cfg.loser_out = loser_out
    cfg.lagged_guiding = lagged_guiding
    return cfg


def workload_request(w, seed, precision=MGFWA_FP32, X=None, y=None, **over):
    """(config, objective buffers) for a workloads.Workload."""
    kw = dict(dim=w.dim, lb=w.lb, ub=w.ub, n_fireworks=w.n_fireworks, sparks_per_firework=w.sparks_per_firework,
              guiding_per_firework=w.guiding_per_firework, eval_budget=w.eval_budget, seed=seed, sigma=w.sigma,
              precision=precision)
    kw.update(over)
    cfg = make_config(**kw)
    if w.kind == MGFWA_OBJ_MLP_CE:
        if X is None:
            import workloads
            X, y = workloads.make_data(w)
        obj = _ObjectiveBuffers(MGFWA_OBJ_MLP_CE, w.widths, w.acts, X, y)
    elif w.kind == MGFWA_OBJ_NET_OUTPUT:
        import workloads
        obj = _ObjectiveBuffers(MGFWA_OBJ_NET_OUTPUT, w.widths, w.acts, params=workloads.make_net(w))
    else:
        obj = _ObjectiveBuffers(MGFWA_OBJ_SPHERE)
    return cfg, obj


def mgfwa_footprint(cfg: mgfwa_config, obj) -> int:
    b = ctypes.c_int64()
    _check(load_library().mgfwa_footprint(ctypes.byref(cfg), ctypes.byref(obj.obj), ctypes.byref(b)))
    return b.value


class Server:
    """Owner of an mgfwa_server_t (see include/mgfwa.h, Serving)."""

    def __init__(self, max_live: int, device_bytes_limit: int):
        h = ctypes.c_void_p()
        _check(load_library().mgfwa_server_create(max_live, device_bytes_limit, ctypes.byref(h)))
        self.handle = h.value
        self.dims = {}

    def submit(self, cfg: mgfwa_config, obj) -> int:
        rid = ctypes.c_int64()
        _check(load_library().mgfwa_server_submit(self.handle, ctypes.byref(cfg), ctypes.byref(obj.obj),
                                                  ctypes.byref(rid)))
        self.dims[rid.value] = cfg.dim
        return rid.value

    def tick(self, generations: int = 1) -> int:
        return load_library().mgfwa_server_tick(self.handle, generations)

    def poll(self, rid: int, want_x: bool = False):
        info = mgfwa_request_info()
        x = np.zeros(self.dims[rid], np.float32) if want_x else None
        _check(load_library().mgfwa_server_poll(self.handle, rid, ctypes.byref(info), _f32p(x)))
        return info, x

    def stats(self) -> mgfwa_server_stats:
        st = mgfwa_server_stats()
        _check(load_library().mgfwa_server_stats_get(self.handle, ctypes.byref(st)))
        return st

    def now(self) -> float:
        return load_library().mgfwa_server_now(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            load_library().mgfwa_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Owner of an mgfwa_group_t over Mgfwa objects (see include/mgfwa.h, Groups); the members must outlive it."""

    def __init__(self, members):
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m.handle for m in self.members])
        h = ctypes.c_void_p()
        _check(load_library().mgfwa_group_create(arr, len(self.members), ctypes.byref(h)))
        self.handle = h.value

    def step(self, n: int = 1) -> int:
        st = load_library().mgfwa_group_step(self.handle, n)
        if st not in (MGFWA_OK, MGFWA_EBUDGET):
            _check(st)
        return st

    def run(self, max_generations: int = 1 << 30, chunk: int = 16) -> None:
        """Step until no member's budget allows another generation."""
        done = 0
        while done < max_generations:
            if self.step(min(chunk, max_generations - done)) == MGFWA_EBUDGET:
                return
            done += chunk

    def close(self):
        if getattr(self, "handle", None):
            load_library().mgfwa_group_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def allgather_reduce_best(key: mgfwa_best_key, group=None) -> mgfwa_best_key:
    """A reduce_best hook body over torch.distributed: gather every rank's key, reduce them with the library's
    host reduction.  Each rank holds one shard of the run."""
    import torch.distributed as dist
    keys = [None] * dist.get_world_size(group)
    dist.all_gather_object(keys, (float(key.f), int(key.shard), int(key.run)), group=group)
    return mgfwa_reduce_best_keys([mgfwa_best_key(f, s, r, 0) for f, s, r in keys])
