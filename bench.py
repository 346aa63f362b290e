"""Throughput of one MGFWA generation on GB300: sparks evaluated per second.

A step is one generation (explosion sampling + mapping, fitness of every
spark, per-firework ranking, multi-guiding sparks + mapping, their fitness,
selection and amplitude update) of the 784-64(ReLU)-10 weight-space workload
(D = 50,890, N = 2048, 5 fireworks x 200 explosion sparks + 8 guiding sparks,
1040 sparks per generation) on synthetic clipped-prototype data.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32]
        python bench.py --impl reference ...   (the CPU oracle on host cores)
Under torchrun each rank runs its own independent run (seed + rank): runs do
not communicate, so scaling is weak and there is no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

import workloads as W

WORKLOAD = W.MLP_784_64_10
METRIC = "sparks evaluated/sec"
UNIT = "sparks/s"


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_seed(rank: int) -> int:
    """Each rank runs its own independent optimisation (weak scaling)."""
    return 1000 + rank


def max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's value (timings are max-reduced over ranks)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Units all ranks processed divided by the slowest rank's time."""
    return world * units_per_rank / seconds


def _capture(kernel: str, source: str):
    """The committed ncu record of `kernel` (profiles/traffic.json), or None when
    the kernel's source changed since that capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(kernel)
    if not rec:
        return None
    sha = hashlib.sha256(open(os.path.join(ROOT, source), "rb").read()).hexdigest()
    if sha != rec.get("sha256"):
        return None
    return rec


def _traffic(kernel: str, source: str):
    """DRAM bytes per launch of `kernel` from the committed ncu capture, or None
    when the kernel's source changed since that capture."""
    rec = _capture(kernel, source)
    if not rec or "dram_bytes_read" not in rec:
        return None
    return rec["dram_bytes_read"] + rec["dram_bytes_write"]


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


def measure_library_peaks():
    """The two peaks the driver's file does not hold, measured the same way (a library GEMM, best of several
    CUDA-event timed calls): dense E4M3 (torch._scaled_mm, 8192^3, BF16 output) and FP32 without tensor cores
    (torch.matmul with TF32 off, 4096^3).  These only serve as roofline denominators.  None where the call is
    unavailable."""
    import torch
    out = {}

    def best_ms(fn, reps):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        return best

    try:
        n = 8192
        A = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        B = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()
        one = torch.ones((), device="cuda", dtype=torch.float32)
        ms = best_ms(lambda: torch._scaled_mm(A, B, scale_a=one, scale_b=one, out_dtype=torch.bfloat16), 10)
        out["fp8_tflops"] = 2 * n ** 3 / (ms / 1e3) / 1e12
        del A, B
    except Exception as e:  # noqa: BLE001 - any failure leaves the derived figure in use
        out["fp8_error"] = f"{type(e).__name__}: {e}"[:160]
    try:
        n = 4096
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        A = torch.randn(n, n, device="cuda")
        B = torch.randn(n, n, device="cuda")
        ms = best_ms(lambda: A @ B, 6)
        torch.backends.cuda.matmul.allow_tf32 = prev
        out["fp32_simt_tflops"] = 2 * n ** 3 / (ms / 1e3) / 1e12
        del A, B
    except Exception as e:  # noqa: BLE001
        out["fp32_error"] = f"{type(e).__name__}: {e}"[:160]
    torch.cuda.empty_cache()
    out["how"] = ("best of 10 torch._scaled_mm E4M3 8192^3 (scales 1, BF16 out) and best of 6 torch.matmul FP32 "
                  "4096^3 with TF32 off, CUDA events, 2 n^3 flop")
    return out


class ClockSampler:
    """SM clock and clock-event reasons sampled while running: read-only NVML queries every 2 ms from a
    thread (through the driver's libnvidia-ml), else nvidia-smi every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits (nvml.h)
    REASON_BITS = (("hw_slowdown", 0x8), ("hw_thermal_slowdown", 0x40), ("sw_thermal_slowdown", 0x20),
                   ("sw_power_cap", 0x4))

    def __init__(self, device_index: int):
        self.proc = None
        self.dev = device_index
        self.samples = []          # (sm MHz, max MHz, reason bits) from NVML
        self.source = None

    def _nvml_start(self):
        import ctypes
        import threading
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        handle = ctypes.c_void_p()
        if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.dev), ctypes.byref(handle)) != 0:
            lib.nvmlShutdown()
            raise OSError("no NVML handle")
        self._lib, self._handle = lib, handle
        self._stop = threading.Event()

        def loop():
            sm, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
            while not self._stop.is_set():
                if (lib.nvmlDeviceGetClockInfo(handle, 1, ctypes.byref(sm)) == 0 and
                        lib.nvmlDeviceGetMaxClockInfo(handle, 1, ctypes.byref(mx)) == 0 and
                        lib.nvmlDeviceGetCurrentClocksEventReasons(handle, ctypes.byref(rs)) == 0):
                    self.samples.append((sm.value, mx.value, rs.value))
                time.sleep(0.002)

        self._thread = threading.Thread(target=loop, daemon=True)
        self._thread.start()
        self.source = "nvml"

    def __enter__(self):
        try:
            self._nvml_start()
            return self
        except (OSError, AttributeError):
            pass
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi"
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.source == "nvml":
            self._stop.set()
            self._thread.join(timeout=5)
            self._lib.nvmlShutdown()
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        if self.source == "nvml":
            for c, m, bits in self.samples:
                sm.append(float(c))
                smax.append(float(m))
                for n, bit in self.REASON_BITS:
                    if bits & bit:
                        reasons.add(n)
        else:
            names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
            for l in getattr(self, "lines", []):
                parts = [p.strip() for p in l.split(",")]
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except (ValueError, IndexError):
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0,
                    "source": self.source}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "source": self.source}


# ---------------------------------------------------------------------------
# The CPU oracle: a bounded sample of the same workload (one firework of the
# five, i.e. 200 explosion + 8 guiding sparks of one generation).

def _oracle_sample_step(orc, prob, p1, seed, gen, fw_x, fw_a, fw_f, threads):
    out = orc.generation(p1, prob, seed, gen, fw_x, fw_a, fw_f, n_threads=threads)
    return out["fw_x"], out["fw_amp"], out["fw_f"], p1.mu * (p1.lam + p1.m)


def cpu_baseline(steps: int = 1, warmup: int = 0):
    import oracle as orc
    threads = os.cpu_count() or 1
    X, y = W.make_data(WORKLOAD)
    prob = orc.Problem.for_workload(WORKLOAD, X, y)
    p1 = orc.params_for(WORKLOAD, mu=1)
    fw_x, fw_a = orc.init(p1, 0)
    fw_f = prob.fitness_many(fw_x, threads).astype(np.float32)
    gen = 0
    for _ in range(warmup):
        gen += 1
        fw_x, fw_a, fw_f, _ = _oracle_sample_step(orc, prob, p1, 0, gen, fw_x, fw_a, fw_f, threads)
    sparks = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        gen += 1
        fw_x, fw_a, fw_f, n = _oracle_sample_step(orc, prob, p1, 0, gen, fw_x, fw_a, fw_f, threads)
        sparks += n
    dt = time.perf_counter() - t0
    return {"value": sparks / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{steps} oracle generation(s) of 1 of the {WORKLOAD.n_fireworks} fireworks ({p1.lam}+{p1.m} "
                      "sparks each) of "
                      f"{WORKLOAD.name}, FP64 fitness, {threads} threads", "seconds": dt}


def oracle_rates():
    """The oracle's rates on the three MLP workloads, single-thread and on every host core, on bounded
    samples (about 10 s in all): the 8-16-3 workload's whole run; the 784-64-10 and 3072-128-64-10
    workloads' fitness of sampled explosion sparks (the generation's dominant cost)."""
    import oracle as orc
    threads = os.cpu_count() or 1
    out = {"cores": threads}
    w0 = W.MLP_8_16_3
    X0, y0 = W.make_data(w0)
    prob0 = orc.Problem.for_workload(w0, X0, y0)
    p0 = orc.params_for(w0)
    r0 = {}
    for key, n in (("single_thread", 1), ("all_cores", threads)):
        t0 = time.perf_counter()
        res = orc.run(p0, prob0, 0, w0.eval_budget, n_threads=n)
        r0[key] = res["evals"] / (time.perf_counter() - t0)
    out[w0.name] = dict(r0, unit=UNIT, sample=f"one whole run ({w0.eval_budget} evaluations)")
    for w, n1, nall in ((W.MLP_784_64_10, 8, 4 * threads), (W.MLP_3072_128_64_10, 1, threads)):
        X, y = W.make_data(w)
        prob = orc.Problem.for_workload(w, X, y)
        p1 = orc.params_for(w, mu=1)
        fw_x, fw_a = orc.init(p1, 0)
        sparks = orc.explode(p1, 0, 1, fw_x, fw_a)
        r = {}
        for key, n, cnt in (("single_thread", 1, n1), ("all_cores", threads, nall)):
            t0 = time.perf_counter()
            prob.fitness_many(sparks[:cnt], n)
            r[key] = cnt / (time.perf_counter() - t0)
        out[w.name] = dict(r, unit=UNIT, sample=f"FP64 fitness of {n1} (one thread) and {nall} (all cores) explosion "
                                                 "sparks of the first generation")
    return out


def reference_arm(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    cb = cpu_baseline(steps=args.steps, warmup=args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * cb["seconds"] / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(args, world),
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def testbed_net(pkg, stream, net_id, steps, **handle_kw):
    """sparks/s of one run on Table 2's network `net_id` (FP32 layers on the CUDA cores), after 3 warm-up
    generations, with the FP32 FLOP rate of its layers."""
    import torch
    w = W.table2_net(net_id)
    w = W.scaled(w, eval_budget=W.budget_for_generations(w.n_fireworks, w.sparks_per_firework,
                                                         w.guiding_per_firework, steps + 5))
    h = pkg.Mgfwa.for_workload(w, 23, stream=stream.cuda_stream, **handle_kw)
    h.step(3)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    h.step(steps)
    b.record(stream)
    torch.cuda.synchronize()
    t = a.elapsed_time(b)
    n = h.info().sparks_per_gen * steps
    h.close()
    sps = n / (t / 1e3)
    prec = {0: "fp32", 3: "fp32x3"}.get(handle_kw.get("precision", 0), str(handle_kw.get("precision")))
    return {"workload": w.name, "value": sps, "unit": UNIT, "ms_per_step": t / steps, "precision": prec,
            "layer_tflops": sps * w.flops_per_spark() / 1e12}


def _config(args, world):
    return {"workload": WORKLOAD.name, "widths": list(WORKLOAD.widths), "dim": WORKLOAD.dim,
            "n_samples": WORKLOAD.n_samples, "fireworks": WORKLOAD.n_fireworks,
            "sparks_per_firework": WORKLOAD.sparks_per_firework,
            "guiding_per_firework": WORKLOAD.guiding_per_firework,
            "sparks_per_generation": WORKLOAD.sparks_per_generation, "runs": world,
            "parallelism": f"independent runs x{world}",
            "l2": (f"working set > L2: {WORKLOAD.sparks_per_generation * WORKLOAD.dim * 4 / 1e6:.1f} MB FP32 sparks + "
                   f"{WORKLOAD.sparks_per_generation * WORKLOAD.widths[0] * WORKLOAD.widths[1] * 2 / 1e6:.1f} MB BF16 "
                   "first-layer operand rewritten every generation")}


# ---------------------------------------------------------------------------

def gpu_arm(args):
    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2501_03944_gb300 as pkg
    pkg.load_library()
    prec = {"bf16": pkg.MGFWA_BF16, "fp32": pkg.MGFWA_FP32, "fp8": pkg.MGFWA_FP8}[args.precision]
    X, y = W.make_data(WORKLOAD)
    seed = run_seed(rank)
    stream = torch.cuda.Stream()
    hbm_peak, bf16_peak, bf16_sus, peak_src = _peaks()
    P = WORKLOAD.sparks_per_generation

    # warm-up, the timed generations, then as many again with per-kernel-group events
    budget_gens = args.warmup + 2 * args.steps + 2
    w = W.scaled(WORKLOAD, eval_budget=W.budget_for_generations(WORKLOAD.n_fireworks, WORKLOAD.sparks_per_firework,
                                                                 WORKLOAD.guiding_per_firework, budget_gens))
    run = pkg.Mgfwa.for_workload(w, seed, precision=prec, X=X, y=y, stream=stream.cuda_stream)
    tile = run.pair_tile()  # the fitness kernel's tile, as the creation-time tuner chose it
    run.step(args.warmup)
    torch.cuda.synchronize()
    launches0 = run.info().kernel_launches
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # the timed region: the production launch path (one graph per generation, programmatic dependent launch)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        run.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = run.info().kernel_launches - launches0
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, dist, "cuda")
    if dist:
        dist.barrier()
    # kernel durations: the next `steps` generations launched kernel by kernel, CUDA events on the
    # handle's stream around each kernel group
    run.profile(True)
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev2.record(stream)
    run.step(args.steps)
    ev3.record(stream)
    torch.cuda.synchronize()
    ms_profiled = ev2.elapsed_time(ev3)
    ktimes = run.kernel_times()
    _, best_f, evals = run.best()
    run.close()

    def timed_generations(handle_kw, steps):
        """sparks/s of `steps` generations of a fresh handle (after 3 warm-up generations)."""
        wk = W.scaled(WORKLOAD, eval_budget=W.budget_for_generations(
            WORKLOAD.n_fireworks, WORKLOAD.sparks_per_firework, WORKLOAD.guiding_per_firework, steps + 5))
        h = pkg.Mgfwa.for_workload(wk, seed + 17, X=X, y=y, stream=stream.cuda_stream, **handle_kw)
        h.step(3)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        h.step(steps)
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b)
        n = h.info().sparks_per_gen * steps
        h.close()
        return {"value": n / (t / 1e3), "ms_per_step": t / steps}

    extra = {}
    if not args.no_extras and world == 1:
        # the serving mix at its arrival rate (an overload: the queue grows) and at a sub-saturating rate,
        # each a bounded window of the trace (--serving-full runs the 2,000-request window)
        extra["serving"] = {"overload": serving_trace(pkg, X, y, n_requests=200, rate_hz=200.0),
                            "sub_saturating": serving_trace(pkg, X, y, n_requests=60, rate_hz=10.0, seed=6)}
        extra["grouped_64_mixed"] = grouped_mixed(pkg)
        extra["fitness_rel_err_vs_fp32"] = fitness_error_vs_fp32(pkg, X, y, stream)
    if not args.no_extras:
        # the plain FP32 one-run path the low-precision path is compared with
        extra["fp32_one_run"] = dict(timed_generations({"precision": pkg.MGFWA_FP32}, 5), precision="fp32")
        # the 3072-128(ReLU)-64(ReLU)-10 network (N = 4096, 8 fireworks x (256 + 8) sparks) in each precision
        extra["mlp3072_128_64_10"] = precision_sweep_3072(pkg, stream)
        X3, y3 = W.make_data(W.MLP_3072_128_64_10)
        extra["mlp3072_128_64_10"]["fitness_rel_err_vs_fp32"] = fitness_error_vs_fp32(
            pkg, X3, y3, stream, n_sparks=64, workload=W.MLP_3072_128_64_10)
        # E4M3 first layer on the tensor cores (elite candidates re-scored in FP32)
        extra["fp8_one_run"] = dict(timed_generations({"precision": pkg.MGFWA_FP8}, max(5, args.steps // 2)),
                                    precision="fp8")
        # the same run with the loser-out tournament (Algorithm 1's step after the selection) on
        extra["loser_out_one_run"] = dict(timed_generations({"precision": prec, "loser_out": 1},
                                                            max(5, args.steps // 2)), precision=args.precision)
        # lagged multi-guiding: explosion and guiding sparks evaluated in one launch from generation 2 on
        extra["lagged_guiding_one_run"] = dict(timed_generations({"precision": prec, "lagged_guiding": 1},
                                                                 max(5, args.steps // 2)), precision=args.precision)
        # the paper's own testbed (Sec. 4.1): Table 2's network 10, its output minimised over its input
        extra["testbed_net10"] = testbed_net(pkg, stream, 10, max(5, args.steps // 2))
        # the same network's layers on the tensor cores at FP32 accuracy (three BF16 parts per operand)
        extra["testbed_net10_fp32x3"] = testbed_net(pkg, stream, 10, max(5, args.steps // 2),
                                                    precision=pkg.MGFWA_FP32X3)
        # the same with lagged multi-guiding: the 40 guiding rows ride in the explosion rows' launches
        extra["testbed_net10_lagged"] = dict(testbed_net(pkg, stream, 10, max(5, args.steps // 2),
                                                         lagged_guiding=1), lagged_guiding=1)
        # 8 independent runs of the same workload in one handle (one fitness launch per generation)
        extra["batched_8_runs"] = dict(timed_generations({"precision": prec, "n_runs": 8}, max(5, args.steps // 2)),
                                       runs=8, precision=args.precision)

    # end to end through the C ABI with host buffers: create (copies X, y from pinned host memory),
    # K generations, best position + FP64 loss back to the host, destroy.
    e2e_s = None
    if not args.no_e2e:
        Xp = torch.from_numpy(X).pin_memory().numpy()
        yp = torch.from_numpy(y).pin_memory().numpy()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run2 = pkg.Mgfwa.for_workload(w, seed + 7919, precision=prec, X=Xp, y=yp, stream=stream.cuda_stream)
        run2.step(args.steps)
        bx2, bf2, ev2 = run2.best()
        run2.close()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")

    lib_peaks = measure_library_peaks() if rank == 0 and world == 1 else {}
    if rank == 0:
        value = whole_job_rate(world, P * args.steps, ms / 1e3)
        e2e_sparks_per_rank = WORKLOAD.n_fireworks + P * args.steps
        # dominant kernel: the explosion-spark fitness launch (mu*lambda sparks per launch)
        fit_ms, fit_n = ktimes["fitness_explosion"]
        n_e = WORKLOAD.n_fireworks * WORKLOAD.sparks_per_firework
        flops = WORKLOAD.flops_per_spark() * n_e
        avg_s = fit_ms / max(fit_n, 1) / 1e3
        kernels = {g: {"ms_total": round(t, 4), "launches": n, "share": round(t / max(ms_profiled, 1e-9), 4)}
                   for g, (t, n) in ktimes.items()}
        if "mlp3072_128_64_10" in extra:
            # the 3072-128-64-10 explosion fitness launch against the burst peak of its operand type
            sw = extra["mlp3072_128_64_10"]
            f8 = lib_peaks.get("fp8_tflops") or 2.0 * bf16_peak
            for name, pk in (("bf16", bf16_peak), ("fp8", f8)):
                if name in sw:
                    sw[name]["fitness_frac_of_burst"] = sw[name]["fitness_tflops"] / pk
                    sw[name]["peak_tflops"] = pk
        # the kernel is timed launch by launch (a few tenths of a millisecond each), so the burst peak is the
        # denominator; the ratio to the sustained (power-capped) peak is reported beside it
        if prec == pkg.MGFWA_BF16:
            roof = {"bound": "tensor", "achieved": flops / avg_s / 1e12, "peak": bf16_peak, "unit": "TFLOP/s",
                    "peak_source": f"{peak_src} bf16 burst (kernel timed launch by launch)"}
            roof["frac_of_sustained"] = roof["achieved"] / bf16_sus
        elif prec == pkg.MGFWA_FP8:
            f8 = lib_peaks.get("fp8_tflops")
            roof = {"bound": "tensor", "achieved": flops / avg_s / 1e12, "unit": "TFLOP/s",
                    "peak": f8 if f8 else 2.0 * bf16_peak,
                    "peak_source": ("measured fp8 burst (torch._scaled_mm E4M3 8192^3)" if f8 else
                                    f"{peak_src} bf16 burst x 2 (the nominal fp8 / bf16 dense ratio)")}
        else:
            f32 = lib_peaks.get("fp32_simt_tflops")
            roof = {"bound": "alu", "achieved": flops / avg_s / 1e12, "unit": "TFLOP/s",
                    "peak": f32 if f32 else 152 * 128 * 2 * 2.07e9 / 1e12,
                    "peak_source": ("measured fp32 without tensor cores (torch.matmul 4096^3, TF32 off)" if f32 else
                                    "derived: 152 SMs x 128 FP32 FMA lanes x 2 flop x 2070 MHz")}
        roof["frac"] = roof["achieved"] / roof["peak"]
        tkey = "k_fitness_pair" + ("" if WORKLOAD is W.MLP_784_64_10 else ":" + WORKLOAD.name)
        roof["traffic"] = (_traffic(tkey, "paper_2501_03944_gb300/csrc/k_fitness_pair.cu")
                           if prec == pkg.MGFWA_BF16 else None)
        roof["traffic_unit"] = "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)"
        roof["kernel"] = (f"fitness of the explosion sparks ({n_e} sparks x {WORKLOAD.n_samples} samples per "
                          "launch)")
        # HBM-bound kernels: algorithmic bytes / time
        D = WORKLOAD.dim
        wd = WORKLOAD.widths
        w1 = wd[0] * wd[1]
        w_later = sum(wd[l] * wd[l + 1] for l in range(1, len(wd) - 1))
        # operand bytes per spark: the first-layer block (BF16 or E4M3) and the BF16 copies of the later
        # layers' weights
        op_b = {pkg.MGFWA_BF16: 2 * w1 + 2 * w_later, pkg.MGFWA_FP8: w1 + 2 * w_later}.get(prec, 0)
        exp_bytes = n_e * (4 * D + op_b)
        # rows each guiding spark reads: its top and bottom subsets, k = round(sigma * lambda / m) each
        g_size = WORKLOAD.sparks_per_firework // WORKLOAD.guiding_per_firework
        k = max(1, min(int(math.floor(WORKLOAD.sigma * g_size + 0.5)), g_size // 2))
        n_g = WORKLOAD.n_fireworks * WORKLOAD.guiding_per_firework
        guide_bytes = n_g * (2 * k * 4 * D + 4 * D + op_b)
        hbm = {}
        for g, b in (("explode", exp_bytes), ("guide", guide_bytes)):
            t, n = ktimes[g]
            if n:
                gbs = b / (t / n / 1e3) / 1e9
                hbm[g] = {"GB/s": round(gbs, 1), "frac": round(gbs / hbm_peak, 4), "bytes_per_launch": b}
        # the sampler's own bound is instruction issue (one warp instruction per cycle per scheduler): its
        # warp instructions per launch from the committed ncu capture of this source, against the issue rate
        # of every scheduler at the SM clock sampled during the timed region
        ex = _capture("k_explode", "paper_2501_03944_gb300/csrc/k_sample.cu")
        if ex and "explode" in hbm and prec == pkg.MGFWA_BF16 and WORKLOAD is W.MLP_784_64_10:
            import torch
            t, n = ktimes["explode"]
            sms = torch.cuda.get_device_properties(0).multi_processor_count
            mhz = clk.summary().get("sm_mhz") or 2070.0
            peak = sms * 4 * mhz * 1e6 / 1e9
            ach = ex["warp_instructions"] / (t / n / 1e3) / 1e9
            hbm["explode"]["issue_roofline"] = {
                "bound": "alu", "achieved": round(ach, 1), "peak": round(peak, 1),
                "unit": "G warp instructions/s", "frac": round(ach / peak, 4),
                "warp_instructions": ex["warp_instructions"],
                "peak_source": f"derived: {sms} SMs x 4 schedulers x 1 warp instruction per cycle x {mhz:.0f} MHz"}
        # the whole generation against its ideal: every spark's fitness at the tensor peak above plus the
        # sampling and guiding bytes at the HBM peak (rank and selection take a few microseconds; the FP32
        # re-score of the elite candidates is accuracy work on top of the metric's and is left out)
        ideal_ms = 1e3 * (WORKLOAD.flops_per_spark() * P / (roof["peak"] * 1e12) +
                          (exp_bytes + guide_bytes) / (hbm_peak * 1e9))
        gen_roof = {"ideal_ms": round(ideal_ms, 4), "ms_per_step": round(ms / args.steps, 4),
                    "frac": round(ideal_ms / (ms / args.steps), 4),
                    "how": "ideal = fitness flops of all sparks / roofline.peak + (explode + guide bytes) / HBM peak"}
        cb = None
        if world == 1 and not args.no_cpu_baseline:
            c = cpu_baseline(steps=3)
            cb = {k2: c[k2] for k2 in ("value", "unit", "cores", "kind", "sample")}
            cb["by_workload"] = oracle_rates()
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {"bf16": "bf16", "fp32": "f32", "fp8": "e4m3"}[args.precision],
                "data": "synthetic", "config": _config(args, world),
                "clocks": clk.summary(), "gpu_launches": launches,
                "e2e": None if e2e_s is None else {
                    "value": whole_job_rate(world, e2e_sparks_per_rank, e2e_s), "unit": UNIT,
                    "h2d_bytes_per_step": (X.nbytes + y.nbytes) / args.steps,
                    "d2h_bytes_per_step": (4 * D + 8) / args.steps,
                    "note": "create (X, y from pinned host) + K generations + best (x, FP64 loss) + destroy"},
                "roofline": roof, "generation_roofline": gen_roof, "hbm_kernels": hbm, "kernels": kernels,
                "fitness_tile": None if tile[0] < 0 else {
                    "sparks_per_tile": tile[0], "stages": tile[1], "k_tail_mmas": tile[3], "tuned": bool(tile[2])},
                "library_peaks": lib_peaks,
                "kernel_timing": {"how": "the next `steps` generations after the timed region, launched kernel by "
                                         "kernel with CUDA events on the handle's stream around each kernel group "
                                         "(roofline.achieved, hbm_kernels and kernels come from it)",
                                  "ms_per_step": ms_profiled / args.steps},
                "best_f_fp64": best_f, "evals": evals, "cpu_baseline": cb, **extra}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def precision_sweep_3072(pkg, stream, gens: int = 3):
    """sparks/s of a few generations of the 3072-128-64-10 workload per precision (after one warm-up
    generation; FP32 takes 2 generations, it is two orders of magnitude slower)."""
    import torch
    w0 = W.MLP_3072_128_64_10
    X3, y3 = W.make_data(w0)
    out = {}
    for name, prec, g in (("bf16", pkg.MGFWA_BF16, gens), ("fp8", pkg.MGFWA_FP8, gens), ("fp32", pkg.MGFWA_FP32, 2)):
        w = W.scaled(w0, eval_budget=W.budget_for_generations(w0.n_fireworks, w0.sparks_per_firework,
                                                              w0.guiding_per_firework, g + 2))
        h = pkg.Mgfwa.for_workload(w, 77, precision=prec, X=X3, y=y3, stream=stream.cuda_stream)
        h.step(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        h.step(g)
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b)
        # one more generation kernel by kernel: the explosion-spark fitness launch's duration
        h.profile(True)
        h.step(1)
        fit_ms, fit_n = h.kernel_times()["fitness_explosion"]
        h.profile(False)
        _, best_f, _ = h.best()
        h.close()
        n_e = w0.n_fireworks * w0.sparks_per_firework
        out[name] = {"sparks_per_s": h.sparks_per_gen * g / (t / 1e3), "ms_per_generation": t / g,
                     "best_f_fp64": best_f, "fitness_launch_ms": fit_ms / max(fit_n, 1),
                     "fitness_tflops": w0.flops_per_spark() * n_e / (fit_ms / max(fit_n, 1) / 1e3) / 1e12}
    return out


def fitness_error_vs_fp32(pkg, X, y, stream, n_sparks: int = 128, workload=None):
    """Relative error of the BF16 and FP8 fitness against the FP32 path on a workload's own explosion
    sparks (generation 4 of a run; the bench workload by default), the qualifier of the throughput metric
    (<= 1e-2)."""
    out = {}
    w = W.scaled(workload or WORKLOAD, eval_budget=10 ** 9)
    for name, prec in (("bf16", pkg.MGFWA_BF16), ("fp8", pkg.MGFWA_FP8)):
        h = pkg.Mgfwa.for_workload(w, 4242, precision=prec, X=X, y=y, stream=stream.cuda_stream)
        h.step(3)
        h.phase(pkg.MGFWA_PHASE_EXPLODE)
        sparks = h.read(pkg.MGFWA_BUF_SPARKS)[:n_sparks]
        for ph in range(pkg.MGFWA_PHASE_EVAL_E, pkg.MGFWA_PHASE_SELECT + 1):
            h.phase(ph)
        low = h.evaluate(sparks, prec).astype(np.float64)
        f32 = h.evaluate(sparks, pkg.MGFWA_FP32).astype(np.float64)
        h.close()
        rel = np.abs(low - f32) / np.abs(f32)
        out[name] = {"max": float(rel.max()), "median": float(np.median(rel)), "sparks": int(n_sparks),
                     "within_1e-2": bool(rel.max() <= 1e-2)}
    return out


def grouped_mixed(pkg, n: int = 64, gens: int = 5, seed: int = 3):
    """64 runs of different shapes (D log-uniform in [195, 50,890] over the MLP families, 3..8 fireworks,
    32..256 sparks, batches of 512..2048; BF16 where the tensor-core path takes the net, else FP32), timed
    end to end (wall clock, synchronised) three ways: one CUDA graph launch per generation for all runs
    (a group), every run's generation launched on its own stream in turn, and one run at a time."""
    import torch
    ws = W.mixed_batch(n, seed, generations=gens + 1)
    data = [W.make_data(w) for w in ws]
    precs = [pkg.MGFWA_BF16 if w.widths[1] == 64 else pkg.MGFWA_FP32 for w in ws]

    def members():
        return [pkg.Mgfwa.for_workload(w, 500 + k, precision=p, X=d[0], y=d[1])
                for k, (w, p, d) in enumerate(zip(ws, precs, data))]

    sparks = gens * sum(w.sparks_per_generation for w in ws)
    out = {"runs": n, "generations": gens, "sparks_per_step": sparks // gens,
           "dims": [int(min(w.dim for w in ws)), int(max(w.dim for w in ws))]}
    hs = members()
    g = pkg.Group(hs)
    g.step(1)  # captures the graph
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.step(gens)
    torch.cuda.synchronize()
    out["graph"] = {"sparks_per_s": sparks / (time.perf_counter() - t0)}
    g.close()
    for h in hs:
        h.close()
    hs = members()
    for h in hs:
        h.step(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(gens):
        for h in hs:
            h.step(1)
    torch.cuda.synchronize()
    out["streams"] = {"sparks_per_s": sparks / (time.perf_counter() - t0)}
    for h in hs:
        h.close()
    hs = members()
    for h in hs:
        h.step(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for h in hs:
        h.step(gens)
        torch.cuda.synchronize()
    out["one_at_a_time"] = {"sparks_per_s": sparks / (time.perf_counter() - t0)}
    for h in hs:
        h.close()
    return out


def serving_trace(pkg, X, y, n_requests: int = 40, rate_hz: float = 200.0, max_live: int = 8, seed: int = 5):
    """Continuous batching on one GPU: Poisson arrivals (mean rate_hz) of optimisation requests drawn
    0.6 / 0.3 / 0.1 from the 8-16(tanh)-3 (FP32: its 16-unit layer is not a tensor-core shape),
    784-64-10 (BF16, FP32 elite re-score) and 3072-128-64-10 (BF16, FP32 elite re-score) workloads, each
    with a budget drawn uniformly in [10k, 100k] evaluations (whole generations).  Latency is from each
    request's arrival to its result; throughput counts every spark."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate_hz, n_requests))
    fams = [(W.MLP_8_16_3, pkg.MGFWA_FP32), (WORKLOAD, pkg.MGFWA_BF16), (W.MLP_3072_128_64_10, pkg.MGFWA_BF16)]
    data = [W.make_data(f[0]) for f in fams]
    data[1] = (X, y)
    reqs, kinds = [], []
    for k in range(n_requests):
        j = int(rng.choice(3, p=[0.6, 0.3, 0.1]))
        w0, prec = fams[j]
        budget = int(rng.uniform(10_000, 100_000))
        gens = max(1, (budget - w0.n_fireworks) // w0.sparks_per_generation)
        w = W.scaled(w0, eval_budget=W.budget_for_generations(w0.n_fireworks, w0.sparks_per_firework,
                                                              w0.guiding_per_firework, gens))
        reqs.append(pkg.workload_request(w, 7000 + k, prec, X=data[j][0], y=data[j][1]))
        kinds.append(j)
    with pkg.Server(max_live=max_live, device_bytes_limit=1 << 36) as s:
        ids, live_samples = [], []
        t0 = s.now()
        nxt = 0
        while True:
            now = s.now() - t0
            while nxt < n_requests and arrivals[nxt] <= now:
                ids.append(s.submit(*reqs[nxt]))
                nxt += 1
            st = s.stats()
            if st.live or st.queued:
                live_samples.append(st.live)
                s.tick(1)
            elif nxt == n_requests:
                break
            else:
                time.sleep(max(0.0, min(1e-3, arrivals[nxt] - now)))
        wall = s.now() - t0
        st = s.stats()
        infos = [s.poll(r)[0] for r in ids]
    lat = np.array([i.t_done - t0 - arrivals[k] for k, i in enumerate(infos)])
    by = {}
    for j, name in enumerate(("mlp8-16-3", "mlp784-64-10", "mlp3072-128-64-10")):
        sel = [k for k in range(n_requests) if kinds[k] == j]
        if sel:
            by[name] = {"requests": len(sel), "latency_ms_p50": round(float(np.percentile(lat[sel], 50)) * 1e3, 2),
                        "latency_ms_p99": round(float(np.percentile(lat[sel], 99)) * 1e3, 2)}
    return {"requests": n_requests, "completed": int(sum(i.state == pkg.MGFWA_REQ_DONE for i in infos)),
            "arrival_rate_hz": rate_hz, "max_live": max_live, "wall_s": round(wall, 4),
            "sparks_per_s": st.sparks_evaluated / wall,
            "latency_ms_p50": round(float(np.percentile(lat, 50)) * 1e3, 3),
            "latency_ms_p99": round(float(np.percentile(lat, 99)) * 1e3, 3),
            "mean_live": round(float(np.mean(live_samples)), 2), "by_workload": by,
            "mix": "0.6 mlp8-16-3 fp32 / 0.3 mlp784-64-10 bf16 / 0.1 mlp3072-128-64-10 bf16; budgets U(10k, 100k) "
                   "evaluations; Poisson arrivals"}


def serving_full(args):
    """The serving workload's full window: 2,000 Poisson requests at 200/s, and 500 at a sub-saturating
    10/s; one JSON line with both (rank 0, one GPU)."""
    import torch
    torch.cuda.set_device(0)
    import paper_2501_03944_gb300 as pkg
    pkg.load_library()
    X, y = W.make_data(WORKLOAD)
    out = {"serving_full": {"overload": serving_trace(pkg, X, y, n_requests=2000, rate_hz=200.0),
                            "sub_saturating": serving_trace(pkg, X, y, n_requests=500, rate_hz=10.0, seed=6)}}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=("gb300", "reference"))
    ap.add_argument("--precision", default="bf16", choices=("bf16", "fp32", "fp8"))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end request (profiling runs)")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP32 and batched comparison runs")
    ap.add_argument("--serving-full", action="store_true",
                    help="only the serving workload's full 2,000-request window (a few minutes)")
    ap.add_argument("--workload", default=W.MLP_784_64_10.name,
                    choices=[w.name for w in (W.MLP_784_64_10, W.MLP_3072_128_64_10, W.MLP_8_16_3)],
                    help="the timed step's workload (the metric is quoted on the 784-64-10 one)")
    ap.add_argument("--fireworks", type=int, default=0,
                    help="override the workload's firework count (smaller profiling captures)")
    args = ap.parse_args()
    global WORKLOAD
    WORKLOAD = W.ALL[args.workload]
    if args.fireworks > 0:
        WORKLOAD = W.scaled(WORKLOAD, n_fireworks=args.fireworks)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_arm(args)
    if args.serving_full:
        return serving_full(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
