#!/usr/bin/env python3
"""Benchmark of the split-step Crank-Nicolson GP step on one GB300 (or N
independent replicas, one per GPU, under torchrun).

    python bench.py [--steps K] [--warmup W] [--workload real_large]
    python bench.py --impl reference ...        # the FP64 CPU oracle, timed

A step is one pass of the whole hot path over the grid: the fused kick +
x line solve, the y line solve, the z line solve with its fused norm, and
(every 10 steps) the observables reduction that tracks norm and energy
drift, queued on the device.  Metric: CN site-updates/s (grid sites x steps
/ seconds).  Prints ONE JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1601_04641_gb300 import inputs, replicas  # noqa: E402

METRIC = "CN site-updates/s"
UNIT = "site-updates/s"
TRACK_EVERY = 10

WORKLOADS = {
    # name: (problem factory, precision, field, real time, g used to prepare the start state)
    "real_large": (inputs.real_large, "f32", "complex", True),
    "real_large_half": (inputs.real_large_half, "f32", "complex", True),
    "real_medium": (inputs.real_medium, "f64", "complex", True),
    "imag_small": (inputs.imag_small, "f64", "real", False),
    "imag_large_real": (inputs.imag_large, "f32", "real", False),
    "imag_large_cplx": (inputs.imag_large, "f32", "complex", False),
    "imag_large_real_half": (inputs.imag_large_half, "f32", "real", False),
    "imag_xl_real": (inputs.imag_xl, "f32", "real", False),
    "imag_xl_f16": (inputs.imag_xl, "f16", "real", False),
}
# batched workloads (run_batch_workload): the 64 uneven condensates, every
# instance active, FP32 complex or real field
BATCH_WORKLOADS = {"batch64_c64": "complex", "batch64_real": "real"}

# FP64 arithmetic of the FP64 complex real-time step, counted from the
# kernels' operations (an FMA is 2 flops, a multiply or add 1): the kick
# 34 per site (scale 2, |q|^2 3, phase 3, sin/cos series 20, rotation 6);
# each line solve 30 per node (right-hand side 10, forward 12, backward 8),
# three of them; the observables 29 per site per call.  The FP64 peak is the
# profiling recipe's nominal 1.25 TFLOP/s (an FMA-chain probe on this part
# measured 1.255).
FP64_FLOPS_STEP_REALTIME = 34 + 3 * 30
FP64_FLOPS_OBSERVABLES = 29
FP64_PEAK_GFLOPS = 1250.0

# DRAM bytes (read + write) per launch from `ncu` of each kernel, with the
# sha256 prefix of the kernel sources they were taken from; a figure whose
# sources have changed since is reported as null.
NCU_TRAFFIC = {
    # ncu --set full of the 480x400x160 half-depth case (profiles/), scaled x2
    # by sites to a full 480x400x320 launch: (read + write) bytes per launch
    ("real_large", "zsweep_norm"): (2 * (246.269440e6 + 200.813568e6), "e8585e1feeacb572"),
    ("real_large", "kick_xsweep"): (2 * (257.253120e6 + 193.859584e6), "e8585e1feeacb572"),
    ("real_large", "ysweep"): (2 * (253.209088e6 + 193.392128e6), "e8585e1feeacb572"),
}


SWEEP_SOURCES = ("gp_internal.h", "gp_host.cu", "gp_sweep.cuh", "gp_sweep_tma.cuh", "k_sweep_inst.cuh")


def kernel_source_hash() -> str:
    """sha256 prefix of the line-solve kernels' sources and of the host code
    that encodes their tensor maps (the kernels whose DRAM traffic
    NCU_TRAFFIC records)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1601_04641_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn in SWEEP_SOURCES or (fn.startswith("k_sweep_") and fn.endswith(".cu")):
            with open(os.path.join(csrc, fn), "rb") as f:
                h.update(f.read())
    return h.hexdigest()[:16]


def guarded(fn):
    """The result of one secondary section of the JSON line, or {"error":
    message} if it raised: a failing section is reported in the line instead
    of losing the headline figures measured before it."""
    try:
        return fn()
    except Exception as e:  # reported in the line
        return {"error": "%s: %s" % (type(e).__name__, e)}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.rows = []
        self.proc = None

    def start(self):
        cmd = ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + ",".join(self.FIELDS),
               "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clocks not sampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in self.rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        power = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        reasons = set()
        for r in self.rows:
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                  "sw_power_cap"), r[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        load = sorted(sm)[len(sm) // 2:] if sm else []
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None,
                "samples": len(self.rows), "reasons": sorted(reasons)}


def gpu_id_for(torch, dev):
    try:
        props = torch.cuda.get_device_properties(dev)
        return "%08X:%02X:%02X.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        first = vis.split(",")[dev] if vis else str(dev)
        return first


# ------------------------------------------------------------------ CPU oracle leg
def host_cpu():
    """Model name (lscpu, else /proc/cpuinfo) and logical CPU count of the host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu model")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"model": model, "logical_cpus": os.cpu_count()}


def _oracle_threads():
    """Threads for the all-core oracle build: every host CPU (set before the
    OpenMP runtime loads)."""
    n = os.cpu_count() or 1
    os.environ["OMP_NUM_THREADS"] = str(n)
    return n


def oracle_rate(problem, realtime, budget_s, threads=1, steps=None):
    """Time the FP64 CPU oracle, as it stands, on a slab of the workload
    (the full y-z planes, fewer x planes) for about `budget_s` seconds:
    the serial build (threads = 1) or the OpenMP build on `threads` cores
    (the kick's sites and the sweeps' lines shared out; sums serial)."""
    import oracle
    nx, ny, nz = problem.shape
    path = oracle.build() if threads == 1 else oracle.build_openmp()
    est_ns = 130.0 / threads
    planes = max(3, min(nx, int(budget_s / (est_ns * 1e-9 * ny * nz * (steps or 2)))))
    shape = (planes, ny, nz)
    psi = inputs.random_field(shape, seed=1)
    with oracle.use_library(path):
        oracle.renormalize(psi, problem.d)
        nsteps = steps or 1
        t0 = time.perf_counter()
        oracle.step(psi, problem.d, problem.dt, problem.omega, problem.g, realtime, nsteps)
        dt = time.perf_counter() - t0
        if steps is None:
            # second pass sized to the budget from the first measurement
            per = dt / (planes * ny * nz)
            nsteps = max(1, int(budget_s / (per * planes * ny * nz)))
            t0 = time.perf_counter()
            oracle.step(psi, problem.d, problem.dt, problem.omega, problem.g, realtime, nsteps)
            dt = time.perf_counter() - t0
    sites = planes * ny * nz
    return {"value": sites * nsteps / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d %s step(s) of a %dx%dx%d slab of the %dx%dx%d grid, FP64 complex, C oracle, %s, "
                      "%.1f s" % (nsteps, "real-time" if realtime else "imaginary-time", planes, ny, nz,
                                  nx, ny, nz, "single-threaded" if threads == 1 else
                                  "OpenMP over sites and lines on %d threads" % threads, dt)}


def cpu_baseline(problem, realtime, budget_s):
    """The oracle on all host cores (the reported baseline) and on one core."""
    n = _oracle_threads()
    allc = oracle_rate(problem, realtime, budget_s, threads=n)
    one = oracle_rate(problem, realtime, budget_s, threads=1)
    allc["host"] = host_cpu()
    allc["single_thread"] = {"value": one["value"], "cores": 1, "sample": one["sample"]}
    return allc


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    factory, prec, field, realtime = WORKLOADS[args.workload]
    p = factory()
    if field == "real":
        realtime = False
    per_step_budget = max(0.05, 150.0 / max(1, args.steps + args.warmup))
    import oracle
    threads = _oracle_threads()
    path = oracle.build_openmp()
    nx, ny, nz = p.shape
    planes = max(3, min(nx, int(per_step_budget / (130e-9 / threads * ny * nz))))
    shape = (planes, ny, nz)
    psi = inputs.random_field(shape, seed=1)
    with oracle.use_library(path):
        oracle.renormalize(psi, p.d)
        for _ in range(args.warmup):
            oracle.step(psi, p.d, p.dt, p.omega, p.g, realtime, 1)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle.step(psi, p.d, p.dt, p.omega, p.g, realtime, 1)
        el = time.perf_counter() - t0
    sites = planes * ny * nz
    value = sites * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": p.name, "grid": list(p.shape),
                       "sample_grid": list(shape), "parallelism": "CPU, OpenMP on %d threads" % threads},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "host": host_cpu(),
                             "sample": "each step: one %s step of a %dx%dx%d slab of the "
                                       "%dx%dx%d grid, FP64 C oracle, OpenMP over sites and lines "
                                       "on %d threads" %
                                       ("real-time" if realtime else "imaginary-time",
                                        planes, ny, nz, nx, ny, nz, threads)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU leg
_GROUND = {}  # (grid, d, trap, g, dt) -> (psi float64 CUDA tensor, info)


def ground_state_of(torch, p, dev):
    """The imaginary-time ground state at the preparation nonlinearity
    g_prepare, dt = 0.1 d^2, converged to |mu(n) - mu(n-10)| < 1e-10 in FP64
    (FP32 real-field dt schedule, then FP64; solver.ground_state), computed
    once per run and kept on the device."""
    from paper_1601_04641_gb300.solver import ground_state
    g_prep = p.meta.get("g_prepare", p.g)
    dt_imag = 0.1 * min(p.d) ** 2
    key = (tuple(p.shape), tuple(p.d), tuple(p.omega), g_prep, dt_imag)
    if key not in _GROUND:
        _GROUND[key] = ground_state(p.shape, p.d, dt_imag, p.omega, g_prep, tol=1e-10, device=dev)
    return _GROUND[key]


def prepare(torch, gp, p, realtime, dev=0):
    """Start state.  Real time: the ground state at g_prepare (reading R8),
    then the quench to g (the handle already holds g and the real-time dt).
    Imaginary time: the Gaussian."""
    if realtime:
        psi, _ = ground_state_of(torch, p, dev)
        gp.set_psi(psi.to(gp.psi.dtype))
    else:
        gp.init_gaussian()
    torch.cuda.synchronize()


def time_workload(torch, name, steps, warmup, dev):
    from paper_1601_04641_gb300.solver import GP
    factory, prec, field, realtime = WORKLOADS[name]
    p = factory()
    gp = GP(p.shape, p.d, p.dt, p.omega, p.g, prec, field, device=dev)
    prepare(torch, gp, p, realtime, dev)
    step = gp.step_real if realtime else gp.step_imag
    gp.set_tracking(TRACK_EVERY, (steps + warmup) // TRACK_EVERY + 4)
    stream = gp.stream
    step(warmup)
    torch.cuda.synchronize()
    res = {"problem": p, "gp": gp, "prec": prec, "field": field, "realtime": realtime}
    res["step"] = step
    return res


def timed_region(torch, res, steps, dist):
    gp, step = res["gp"], res["step"]
    stream = gp.stream
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    step(steps)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    e1.synchronize()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    return e0.elapsed_time(e1) / 1e3


def kernel_breakdown(torch, res, steps):
    """Average duration of each kernel of the step, from CUDA events recorded
    between the stages on the launching stream."""
    gp = res["gp"]
    rt = res["realtime"]
    stream = gp.stream
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    torch.cuda.synchronize()
    for s in range(steps):
        ev[s][0].record(stream)
        for stage in range(3):
            gp.stage(stage, rt)
            ev[s][stage + 1].record(stream)
    torch.cuda.synchronize()
    names = ["kick_xsweep", "ysweep", "zsweep_norm"]
    out = {}
    for stage in range(3):
        ms = [ev[s][stage].elapsed_time(ev[s][stage + 1]) for s in range(steps)]
        out[names[stage]] = sum(ms) / len(ms) / 1e3
    return out


def e2e_region(torch, res, steps, dist):
    """Through the public API with host buffers: psi uploaded from pinned host
    memory, `steps` steps with the observables read back to the host every 10
    steps, psi downloaded to pinned host memory -- all inside the timed region."""
    import numpy as np
    gp, step = res["gp"], res["step"]
    host = torch.empty(gp.shape, dtype=gp.psi.dtype, pin_memory=True)
    host.copy_(gp.psi.cpu())
    out = torch.empty_like(host).pin_memory()
    src = host.numpy()
    dst = out.numpy()
    gp.set_tracking(0, 0)
    n_obs = 0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gp.lib.gp_set_psi(gp.h, src.ctypes.data_as(ctypes.c_void_p), 0)
    done = 0
    while done < steps:
        n = min(TRACK_EVERY, steps - done)
        step(n)
        done += n
        gp.observables()
        n_obs += 1
    gp.lib.gp_get_psi(gp.h, dst.ctypes.data_as(ctypes.c_void_p), 0)
    el = time.perf_counter() - t0
    if dist:
        dist.barrier()
    nbytes = host.numel() * host.element_size()
    obs_bytes = 16 * 8 * n_obs
    return el, nbytes / steps, (nbytes + obs_bytes) / steps


def precision_vs_fp64(torch, dev, steps):
    """Accuracy of the complex64 form on the benchmark workload: the same
    500-step quench run in FP64 from the same (FP32-representable) start
    state; errors of mu, E, rms and psi (relative L2) of the FP32 run.  At
    61 M sites the C oracle would need most of an hour, so the reference is
    the FP64 GPU path, which the tests hold to the oracle within 1e-12."""
    from paper_1601_04641_gb300.solver import GP
    p = inputs.real_large()
    g64 = GP(p.shape, p.d, p.dt, p.omega, p.g, "f64", "complex", device=dev)
    psi0, info = ground_state_of(torch, p, dev)
    start = psi0.to(torch.complex64)
    g64.set_psi(start.to(torch.complex128))
    g32 = GP(p.shape, p.d, p.dt, p.omega, p.g, "f32", "complex", device=dev)
    g32.set_psi(start)
    del start
    # the reductions alone: the same complex64 values summed by the complex64
    # kernel (FP32 per thread with compensation, FP64 across blocks) and by
    # the FP64 kernel (FP64 throughout)
    r64, r32 = g64.observables(), g32.observables()
    reduction = {k: abs(r32[k] - r64[k]) / abs(r64[k]) for k in ("norm", "mu", "energy", "rms_x", "rms_y", "rms_z")}
    g64.step_real(steps)
    g32.step_real(steps)
    o64, o32 = g64.observables(), g32.observables()
    a = g64.get_psi(as_numpy=False)
    b = g32.get_psi(as_numpy=False).to(torch.complex128)
    rel_l2 = float(torch.linalg.vector_norm(b - a) / torch.linalg.vector_norm(a))
    del a, b
    g64.close()
    g32.close()
    torch.cuda.synchronize()
    rel = lambda k: abs(o32[k] - o64[k]) / abs(o64[k])
    return {"workload": p.name, "steps": steps, "reference": "FP64 GPU path from the same start state",
            "start": {"state": "imaginary-time ground state at g %g, dt 0.1 d^2 (FP32 real-field dt schedule, "
                               "then FP64 to |dmu| < %g between checks 10 steps apart), rounded to complex64, "
                               "quenched to g %g" % (p.meta["g_prepare"], info["tol"], p.g),
                      "mu": info["mu"], "last_dmu": info["last_dmu"], "fp32_schedule_steps": info["fp32_schedule_steps"],
                      "fp64_steps": info["fp64_steps"], "prepare_s": info["fp32_s"] + info["fp64_s"]},
            "mu_rel_err": rel("mu"), "energy_rel_err": rel("energy"),
            "rms_rel_err": [rel("rms_x"), rel("rms_y"), rel("rms_z")], "norm_rel_err": rel("norm"),
            "psi_rel_l2": rel_l2, "bounds": {"mu_rel": 1e-5, "psi_rel_l2": 1e-4},
            "reduction_fp32_compensated_vs_fp64": reduction}


def symmetric_splitting(torch, dev, steps, warmup):
    """Both splittings of the real-time step: first order (kick, sweeps; the
    main line) and symmetric (half kick, sweeps, half kick; records every
    TRACK_EVERY steps settle the pending half kick).
    - speed: the benchmark workload from the same prepared state, time per
      step with tracking;
    - accuracy: the FP64 240x200x160 workload over 200 steps of its dt, the
      relative L2 distance of psi from a symmetric-splitting run at dt/8
      (whose own error is about 1/64 of the symmetric one at dt)."""
    out = {"speed": {"workload": None, "steps": steps}}
    for order in (1, 2):
        res = time_workload(torch, "real_large", steps, 0, dev)
        gp = res["gp"]
        gp.set_splitting(order)
        gp.set_tracking(TRACK_EVERY, steps // TRACK_EVERY + 4)
        gp.step_real(warmup)
        el = timed_region(torch, res, steps, None)
        gp.close()
        out["speed"]["workload"] = res["problem"].name
        out["speed"]["order_%d" % order] = {"ms_per_step": 1e3 * el / steps,
                                            "value": res["problem"].sites * steps / el, "unit": UNIT}
    from paper_1601_04641_gb300.solver import GP
    p = inputs.real_medium()
    runs = {}
    for name, order, sub in (("order_1", 1, 1), ("order_2", 2, 1), ("reference", 2, 8)):
        gp = GP(p.shape, p.d, p.dt / sub, p.omega, p.g, "f64", "complex", device=dev)
        prepare(torch, gp, p, True, dev)
        gp.set_splitting(order)
        gp.step_real(200 * sub)
        runs[name] = gp.get_psi(as_numpy=False)
        gp.close()
    ref = runs.pop("reference")
    out["accuracy"] = {"workload": "%s, 200 steps of dt %g, FP64" % (p.name, p.dt),
                       "rel_l2_vs_dt_over_8": {k: float(torch.linalg.vector_norm(v - ref) /
                                                        torch.linalg.vector_norm(ref))
                                               for k, v in runs.items()}}
    return out


# Final level of the dt schedules: |dmu| < tol * SCHEDULE_FINAL with stop rule
# 2.  A schedule's last level starts at the fixed point of a coarser dt, from
# which mu and E approach along several modes at once and can pass through a
# sign change of their differences; the tighter final level and the
# two-check rule end its runs no farther from mu* than the plain method's
# (measured on the 64-condensate workload: largest error 1.1e-5 against the
# plain method's 5.5e-5; at tol/10, 7.7e-5).  The FP32 batch at dt alone ends
# slightly farther than the plain FP64 method at the same tol (6.3e-5) and
# runs to tol * BATCH_DT_FINAL with rule 2 for the matched comparison (2.1e-5).
SCHEDULE_FINAL = 0.03
BATCH_DT_FINAL = 1.0 / 3.0


def schedule_levels(tol):
    return [(10.0, 100 * tol), (3.0, 10 * tol), (1.0, SCHEDULE_FINAL * tol)]


def mu_reference(torch, dev, probs):
    """mu* of every condensate: FP64 batched imaginary time through a dt
    schedule to |dmu|, |dE| < 1e-12 (not part of any timed method)."""
    from paper_1601_04641_gb300.solver import Batch
    b = Batch(probs, "f64", "real", device=dev)
    b.set_stop_rule(1)
    b.init_gaussian()
    b.run_imag_schedule([(10.0, 1e-9), (3.0, 1e-11), (1.0, 1e-12)], 10, 800000)
    mus = [o["mu"] for o in b.observables()]
    b.close()
    return mus


def mu_errors(mus, mustar):
    e = sorted(abs(m - r) / r for m, r in zip(mus, mustar))
    return {"max": e[-1], "median": e[len(e) // 2]}


def batch_step_roofline(torch, dev, probs, field, peak, steps=400):
    """ms per imaginary-time step of the batch with every instance active, and
    its HBM fraction (3 sweeps x read + write of psi: 6 s bytes per site)."""
    from paper_1601_04641_gb300.solver import Batch
    b = Batch(probs, "f32", field, device=dev)
    b.init_gaussian()
    b.step_imag(40)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step_imag(steps)
    e1.record(b.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    tma = b.tma_count()
    b.close()
    sites = sum(p.sites for p in probs)
    elem = 8 if field == "complex" else 4
    gbs = 6 * elem * sites / (ms * 1e-3) / 1e9
    return {"ms_per_step": ms, "achieved_gbs": gbs, "hbm_frac": gbs / peak, "tma_instances": tma,
            "bytes_per_site": 6 * elem}


def time_to_ground_state(torch, dev, count, tol, peak, max_steps=20000):
    """The 64-condensate workload (uneven grids, traps, g) to the ground
    state, each method from the Gaussian, timed from creation to the stop:
    - plain: FP64, one condensate at a time, |mu(n) - mu(n-10)| < tol (the
      plain FP64 GPU method; its distance from mu* sets the accuracy bar);
    - the same FP64 method as one batch;
    - FP32 complex batch, same rule;
    - FP32 batch through the dt schedule (complex and real field).
    Every method's error is measured against mu* (mu_reference) on all
    instances; a speed-up is reported only where the method's largest error
    is no larger than the plain method's."""
    from paper_1601_04641_gb300.solver import GP, Batch
    probs = inputs.batch_problems(count, seed=0)
    sites = sum(p.sites for p in probs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mustar = mu_reference(torch, dev, probs)
    t_ref = time.perf_counter() - t0
    runs = {}

    def batch_run(name, prec, field, levels, rule, tol_run=tol):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b = Batch(probs, prec, field, device=dev)
        b.set_stop_rule(rule)
        b.init_gaussian()
        st = b.run_imag_schedule(levels, 10, max_steps) if levels else b.run_imag_until(tol_run, 10, max_steps)
        mus = [o["mu"] for o in b.observables()]
        torch.cuda.synchronize()
        runs[name] = {"s": time.perf_counter() - t0, "steps_max": max(st), "steps_total": sum(st),
                      "converged": sum(x < max_steps * (len(levels) if levels else 1) for x in st),
                      "mu_err_vs_converged": mu_errors(mus, mustar), "mu": mus}

    t_plain, steps_p, mu_p = 0.0, [], []
    for p in probs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gp = GP(p.shape, p.d, p.dt, p.omega, p.g, "f64", "real", device=dev)
        gp.init_gaussian()
        steps_p.append(gp.run_imag_until(tol, 10, max_steps))
        mu_p.append(gp.observables()["mu"])
        torch.cuda.synchronize()
        t_plain += time.perf_counter() - t0
        gp.close()
    runs["plain_fp64"] = {"s": t_plain, "steps_max": max(steps_p), "steps_total": sum(steps_p),
                          "converged": sum(x < max_steps for x in steps_p),
                          "mu_err_vs_converged": mu_errors(mu_p, mustar), "mu": mu_p}
    batch_run("plain_fp64_batched", "f64", "real", None, 0)
    batch_run("batched_fp32", "f32", "complex", None, 0)
    batch_run("batched_fp32_tight", "f32", "complex", None, 2, tol * BATCH_DT_FINAL)
    levels = schedule_levels(tol)
    batch_run("schedule_fp32", "f32", "complex", levels, 2)
    batch_run("schedule_fp32_real_field", "f32", "real", levels, 2)
    bar = runs["plain_fp64"]["mu_err_vs_converged"]["max"]
    out = {"workload": "%d uneven condensates (seed 0), imaginary time from the Gaussian; stop rule "
                       "|dmu| < %g between checks 10 steps apart" % (count, tol),
           "sites_total": sites,
           "mu_reference": "FP64 batch, dt schedule to |dmu|, |dE| < 1e-12 (%.1f s, untimed)" % t_ref,
           "schedule_levels": "10 dt to %g, 3 dt to %g, dt to %g; stop rule 2 (|dmu| and |dE| below "
                              "the level's tolerance at two consecutive checks)" % tuple(l[1] for l in levels),
           "batched_fp32_tight": "dt alone to |dmu| < %g, stop rule 2" % (tol * BATCH_DT_FINAL),
           "accuracy_bar": {"plain_fp64_max_rel_err": bar}}
    for name, r in runs.items():
        err = r["mu_err_vs_converged"]
        matched = err["max"] <= bar
        out[name] = {k: v for k, v in r.items() if k != "mu"}
        out[name]["matched_accuracy"] = matched
        out[name]["speedup_vs_plain"] = t_plain / r["s"] if matched else None
    out["mu_rel_diff_max_real_vs_complex_field"] = max(
        abs(a - c) / c for a, c in zip(runs["schedule_fp32_real_field"]["mu"], runs["schedule_fp32"]["mu"]))
    out["step_all_active"] = {"complex64": batch_step_roofline(torch, dev, probs, "complex", peak),
                              "float32_real": batch_step_roofline(torch, dev, probs, "real", peak)}
    return out, mustar, bar


def warm_start(torch, dev, n_train, n_held, steps, mustar64=None, bar64=None, tol=1e-7):
    """The learned warm start on 128x96x80 condensates: targets are the
    method's own ground states (FP32 real-field batches through a dt schedule
    and then at dt to |dmu| < 1e-9, where the FP32 iteration settles at its
    fixed point, then 100 FP64 steps), GPU training of the network, then
    imaginary time (FP32 real-field batches) to |dmu|, |dE| < tol on held-out
    parameters from the Gaussian and from the network's prediction (energy
    fallback)."""
    import numpy as np
    from paper_1601_04641_gb300 import warmstart as W
    shape = (128, 96, 80)
    tp = [inputs.sized_box(shape, p.omega, p.g) for p in inputs.batch_problems(n_train, seed=1, g_max=500.0)]
    hp = [inputs.sized_box(shape, p.omega, p.g) for p in inputs.batch_problems(n_held, seed=2, g_max=500.0)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    data, offs, pmax, _, gs_info = W.ground_states(tp, 1e-9, max_steps=60000, device=dev, polish=100,
                                                   with_info=True)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = W.Net(seed=0, device=dev)
    net.set_data(tp, data, offs, pmax)
    t0 = time.perf_counter()
    losses = W.train(net, steps, points=32768, lr=(3e-3, 1e-4))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    max_steps = 60000
    r = W.run_from_starts(net, hp, tol, precision="f32", field="real", max_steps=max_steps, device=dev)
    ttgs = schedule_from_starts(torch, dev, net, 64, 1e-6, mustar64, bar64)
    net.close()
    del data
    sg = np.array(r["steps_gauss"], dtype=float)
    sn = np.array(r["steps_nn"], dtype=float)
    both = (sg < max_steps) & (sn < max_steps)  # the stop rule fired for both starts
    ratio = sg[both] / sn[both]
    mu_rel = [abs(a - b) / abs(a) for a, b, ok in zip(r["mu_gauss"], r["mu_nn"], both) if ok]
    # forward + backward multiply-adds per sample point of the 16-64-64-64-1 net
    macs = (16 * 64 + 64 * 64 + 64 * 64 + 64) * 2 + (64 * 64 + 64 * 64 + 64)
    return {"workload": "128x96x80 condensates, gamma,nu,lambda ~ U[0.5,3], log g ~ U[0, ln 500]; "
                        "%d training ground states (FP32 real-field batches, dt schedule then dt to "
                        "|dmu| < 1e-9, then 100 FP64 steps), %d held-out, FP32 real-field batches in "
                        "imaginary time to |dmu| < %g and |dE| < %g (at most %d steps)" % (n_train, n_held, tol,
                                                                                         tol, max_steps),
            "targets": gs_info,
            "data_s": t_data, "train_s": t_train, "train_steps": steps, "final_loss": losses[-1],
            "train_tflops": 2.0 * macs * 32768 * steps / t_train / 1e12,
            "converged": {"gauss": int((sg < max_steps).sum()), "nn": int((sn < max_steps).sum()),
                          "of": len(hp)},
            "steps_ratio_gauss_over_nn": {"median": float(np.median(ratio)), "mean": float(ratio.mean()),
                                          "min": float(ratio.min()), "max": float(ratio.max())},
            "steps_total": {"gauss": int(sg.sum()), "nn": int(sn.sum())},
            "time_gauss_s": r["time_gauss_s"], "time_nn_s": r["time_nn_s"],
            "time_speedup": r["time_gauss_s"] / r["time_nn_s"], "fallbacks": int(sum(r["fallback"])),
            "mu_rel_diff_max": max(mu_rel) if mu_rel else None,
            "time_to_ground_state_64": ttgs}


def schedule_from_starts(torch, dev, net, count, tol, mustar=None, bar=None, max_steps=20000):
    """The 64-condensate workload, batched FP32, from the Gaussian and from
    the network's prediction (energy fallback to the Gaussian per instance),
    each either through the dt schedule (schedule_levels, stop rule 2) or at
    dt alone (|dmu|, |dE| < tol, stop rule 1); each run timed from batch
    creation to convergence, prediction and fallback test included.  With
    mu* and the plain method's error bar, each run's error is reported and
    the comparison uses only runs within the bar."""
    from paper_1601_04641_gb300.solver import Batch
    probs = inputs.batch_problems(count, seed=0)
    levels = schedule_levels(tol)
    runs = {}
    for start in ("gauss", "nn"):
        for method in ("schedule", "dt"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b = Batch(probs, "f32", "complex", device=dev)
            b.set_stop_rule(2 if method == "schedule" else 1)
            b.init_gaussian()
            fallbacks = 0
            if start == "nn":
                e_gauss = [o["energy"] for o in b.observables()]
                # the Gaussian starts kept on the device (copies through the C ABI)
                keep = [torch.empty(p.shape, dtype=torch.complex64, device="cuda") for p in probs]
                for i, k in enumerate(keep):
                    b._ck(b.lib.gp_batch_get_psi(b.h, i, ctypes.c_void_p(k.data_ptr()), 1))
                net.predict_batch(b)
                e_nn = [o["energy"] for o in b.observables()]
                for i, (en, eg) in enumerate(zip(e_nn, e_gauss)):
                    if not (math.isfinite(en) and en <= eg):
                        b._ck(b.lib.gp_batch_set_psi(b.h, i, ctypes.c_void_p(keep[i].data_ptr()), 1))
                        fallbacks += 1
                del keep
            if method == "schedule":
                steps = b.run_imag_schedule(levels, 10, max_steps)
            else:
                steps = b.run_imag_until(tol, 10, max_steps)
            mus = [o["mu"] for o in b.observables()]
            torch.cuda.synchronize()
            runs[start + "_" + method] = {"s": time.perf_counter() - t0, "steps_total": int(sum(steps)),
                                          "steps_max": int(max(steps)), "mu": mus, "fallbacks": fallbacks}
            b.close()
    out = {"workload": "%d uneven condensates (seed 0), batched FP32 complex; schedule: %s, stop rule 2; "
                       "dt alone: |dmu|, |dE| < %g" % (count, ", ".join("%g dt to %g" % l for l in levels), tol)}
    for name, r in runs.items():
        out[name] = {"s": r["s"], "steps_total": r["steps_total"], "steps_max": r["steps_max"]}
        if mustar:
            err = mu_errors(r["mu"], mustar)
            out[name]["mu_err_vs_converged"] = err
            out[name]["matched_accuracy"] = bar is not None and err["max"] <= bar
    out["fallbacks"] = runs["nn_dt"]["fallbacks"]
    ok = lambda n: (not mustar) or out[n]["matched_accuracy"]
    best_g = min([runs[n]["s"] for n in ("gauss_schedule", "gauss_dt") if ok(n)] or [float("nan")])
    best_n = min([runs[n]["s"] for n in ("nn_schedule", "nn_dt") if ok(n)] or [float("nan")])
    out["best_nn_over_best_gauss"] = best_g / best_n
    out["prediction_helps_schedule"] = runs["gauss_schedule"]["s"] / runs["nn_schedule"]["s"]
    out["prediction_helps_dt"] = runs["gauss_dt"]["s"] / runs["nn_dt"]["s"]
    return out


def time_to_ground_state_sharded(torch, dev, count, tol, rank, world, dist, max_steps=20000):
    """The 64-condensate workload split over the ranks (each rank's batch a
    balanced share by sites, no exchange): wall time of the slowest rank,
    batched FP32 from the Gaussian and through the dt schedule."""
    from paper_1601_04641_gb300.solver import Batch
    probs = inputs.batch_problems(count, seed=0)
    mine = [probs[i] for i in replicas.shard_by_sites([p.sites for p in probs], rank, world)]
    out = {}
    for name, levels in (("batched_fp32_s", None), ("schedule_fp32_s", schedule_levels(tol))):
        torch.cuda.synchronize()
        dist.barrier()
        t0 = time.perf_counter()
        b = Batch(mine, "f32", "complex", device=dev)
        if levels:
            b.set_stop_rule(2)
        b.init_gaussian()
        steps = b.run_imag_schedule(levels, 10, max_steps) if levels else b.run_imag_until(tol, 10, max_steps)
        torch.cuda.synchronize()
        out[name] = replicas.max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        out[name.replace("_s", "_steps_max")] = max(replicas.gather_to_rank0(max(steps), dist) or [0])
        b.close()
    out.update({"workload": "%d uneven condensates (seed 0), imaginary time to |dmu| < %g" % (count, tol),
                "ranks": world, "scaling": "strong (instances shared out by sites)"})
    return out


def run_batch_workload(args):
    """The 64-condensate batch (seed 0) with every instance active: W warm-up
    steps, then K imaginary-time steps timed with CUDA events inside the
    NVTX range "timed" (the profiling case of the batched kernels).  One JSON
    line: site-updates/s and the HBM fraction of 6 s bytes per site."""
    import torch
    from paper_1601_04641_gb300 import build as B
    from paper_1601_04641_gb300.solver import Batch
    B.build()
    torch.cuda.set_device(0)
    field = BATCH_WORKLOADS[args.workload]
    probs = inputs.batch_problems(64, seed=0)
    sites = sum(p.sites for p in probs)
    b = Batch(probs, "f32", field, device=0)
    b.init_gaussian()
    b.step_imag(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(b.stream)
    b.step_imag(args.steps)
    e1.record(b.stream)
    torch.cuda.nvtx.range_pop()
    e1.synchronize()
    el = e0.elapsed_time(e1) / 1e3
    elem = 8 if field == "complex" else 4
    peak, kind = load_peaks()
    print(json.dumps({"metric": METRIC, "value": sites * args.steps / el, "unit": UNIT, "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
                      "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "64 uneven condensates (seed 0), imaginary time, FP32 %s field, "
                                             "all active" % field, "sites": sites,
                                 "tma_instances": b.tma_count()},
                      "hbm_frac": 6 * elem * sites * args.steps / el / 1e9 / peak}), flush=True)
    b.close()
    return 0


def run_ours(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = tdist
    torch.cuda.set_device(local)
    from paper_1601_04641_gb300 import build as B
    B.build()

    res = time_workload(torch, args.workload, args.steps, args.warmup, local)
    p = res["problem"]
    clocks = ClockSampler(gpu_id_for(torch, local))
    clocks.start()
    el = timed_region(torch, res, args.steps, dist)
    clocks.stop()
    el = replicas.max_over_ranks(el, dist, "cuda")
    sites = p.sites
    value = sites * args.steps * world / el
    launches = 3 * args.steps + (args.steps // TRACK_EVERY)
    track = res["gp"].tracking()

    kb = kernel_breakdown(torch, res, min(args.steps, 200))
    top = max(kb, key=kb.get)
    elem = {"f16": 4, "f32": 8, "f64": 16}[res["prec"]]
    if res["field"] == "real":
        elem //= 2
    alg_bytes = 2 * elem * sites  # each kernel reads and writes psi once
    peak, peak_kind = load_peaks()
    achieved = alg_bytes / kb[top] / 1e9
    src_hash = kernel_source_hash()
    tr = NCU_TRAFFIC.get((args.workload, top))
    traffic = tr[0] if tr and tr[1] == src_hash else None

    e2e_el, h2d, d2h = e2e_region(torch, res, args.steps, dist)
    if dist:
        t = torch.tensor([e2e_el], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_el = float(t.item())

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": res["prec"], "data": "synthetic",
        "config": {"workload": p.name, "grid": list(p.shape), "sites": sites,
                   "psi": {"f32": "complex64", "f64": "complex128"}[res["prec"]]
                   if res["field"] == "complex" else {"f16": "float16", "f32": "float32", "f64": "float64"}[res["prec"]],
                   "reductions": "fp64", "dt": p.dt, "g": p.g, "omega": list(p.omega),
                   "track_every": TRACK_EVERY,
                   "l2": ("inputs larger than L2 (psi %.0f MB > 129 MB)" if elem * sites > 129e6 else
                          "psi %.0f MB fits in the 129 MB L2 (no flush: a timing of L2-resident data)") %
                         (elem * sites / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": peak_kind,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "kernel_ms": {k: 1e3 * v for k, v in kb.items()}},
        "e2e": {"value": sites * args.steps * world / e2e_el, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "clocks": clocks.summary(),
        "gpu_launches": launches,
        "drift": {"norm": track[-1]["norm"] - track[0]["norm"] if track else None,
                  "energy_rel": (track[-1]["energy"] - track[0]["energy"]) / track[0]["energy"]
                  if track else None},
    }
    res["gp"].close()

    def also_workload(name):
        """One secondary workload: its step time and per-kernel HBM fractions."""
        r2 = time_workload(torch, name, args.also_steps, 3, local)
        el2 = timed_region(torch, r2, args.also_steps, None)
        kb2 = kernel_breakdown(torch, r2, min(args.also_steps, 50))
        p2 = r2["problem"]
        elem2 = {"f16": 4, "f32": 8, "f64": 16}[r2["prec"]] // (2 if r2["field"] == "real" else 1)
        bytes2 = 2 * elem2 * p2.sites  # algorithmic bytes per sweep launch
        if r2["prec"] == "f64" and r2["field"] == "complex" and r2["realtime"]:
            # FP64 is bound by the FP64 units, not by HBM: flops against the FP64 peak
            flops = p2.sites * (FP64_FLOPS_STEP_REALTIME + FP64_FLOPS_OBSERVABLES / TRACK_EVERY)
            gflops = flops * args.also_steps / el2 / 1e9
            alu = {"bound": "alu", "flops_per_site_step": flops / p2.sites,
                   "achieved_gflops": gflops, "peak_gflops": FP64_PEAK_GFLOPS,
                   "peak_source": "recipe nominal FP64", "alu_frac": gflops / FP64_PEAK_GFLOPS}
        else:
            alu = None
        out = {"workload": p2.name, "grid": list(p2.shape),
               "psi": {(2, "real"): "float16", (4, "real"): "float32", (8, "real"): "float64",
                       (8, "complex"): "complex64",
                       (16, "complex"): "complex128"}[(elem2, r2["field"])],
               "time": "real" if r2["realtime"] else "imaginary",
               "value": p2.sites * args.also_steps / el2,
               "ms_per_step": 1e3 * el2 / args.also_steps, "dtype": r2["prec"],
               "kernel_ms": {k: 1e3 * v for k, v in kb2.items()},
               "kernel_hbm_frac": {k: bytes2 / v / 1e9 / peak for k, v in kb2.items()},
               "step_hbm_frac": 3 * bytes2 * args.also_steps / el2 / 1e9 / peak}
        if alu:
            out["fp64_roofline"] = alu
        if r2["realtime"]:
            _, info = ground_state_of(torch, p2, local)
            out["start"] = {"mu": info["mu"], "last_dmu": info["last_dmu"]}
        o2 = r2["gp"].observables()
        out["mu"] = o2["mu"]
        r2["gp"].close()
        return out

    if args.also and world == 1:
        line["also"] = {name: guarded(lambda: also_workload(name))
                        for name in args.also.split(",") if name and name != args.workload}
    # single-rank sections are guarded; the sharded one is not (a rank that
    # skipped its collectives would leave the others waiting)
    if args.precision and world == 1:
        line["precision_vs_fp64"] = guarded(lambda: precision_vs_fp64(torch, local, 500))
    if args.strang and world == 1:
        line["symmetric_splitting"] = guarded(
            lambda: symmetric_splitting(torch, local, min(args.steps, 500), args.warmup))
    mustar64 = bar64 = None
    if args.gs and world == 1:
        out = guarded(lambda: time_to_ground_state(torch, local, args.gs, 1e-6, peak))
        if isinstance(out, tuple):
            line["time_to_ground_state"], mustar64, bar64 = out
        else:
            line["time_to_ground_state"] = out
    elif args.gs:
        line["time_to_ground_state"] = time_to_ground_state_sharded(torch, local, args.gs, 1e-6, rank, world, dist)
    if args.ws_train and world == 1:
        line["warm_start"] = guarded(
            lambda: warm_start(torch, local, args.ws_train, args.ws_held, args.ws_steps,
                               mustar64 if args.gs == 64 else None, bar64 if args.gs == 64 else None))
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = guarded(lambda: cpu_baseline(p, res["realtime"], args.cpu_budget))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + sorted(BATCH_WORKLOADS), default="real_large")
    ap.add_argument("--also", default="real_medium,imag_large_real,imag_large_cplx,imag_xl_real,imag_xl_f16",
                    help="comma-separated secondary workloads timed after the main one")
    ap.add_argument("--also-steps", type=int, default=200)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--gs", type=int, default=64,
                    help="condensates in the time-to-ground-state comparison (0: skip)")
    ap.add_argument("--ws-train", type=int, default=2000,
                    help="training ground states of the warm-start comparison (0: skip)")
    ap.add_argument("--ws-held", type=int, default=200, help="held-out condensates")
    ap.add_argument("--ws-steps", type=int, default=8000, help="Adam steps")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--strang", type=int, default=1, help="1: also time the symmetric splitting")
    ap.add_argument("--precision", type=int, default=1,
                    help="1: also measure the complex64 run's error against FP64 (500 steps)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        if args.workload in BATCH_WORKLOADS:
            ap.error("the reference arm times the single-condensate workloads")
        return run_reference(args)
    if args.workload in BATCH_WORKLOADS:
        return run_batch_workload(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
