#!/usr/bin/env python
"""Benchmark of the fused finite-volume RK3 step (libjf) on one or more GPUs.

Default workload: compressible Taylor-Green vortex, 256^3 cells, FP32,
Navier-Stokes (WENO5-JS + HLLC + C4 viscous and heat fluxes), TVD-RK3 with the
CFL step computed on the device every step.  One "step" is one full RK3 step
over the whole grid: the CFL reduction and the three stage launches, each
called through the C ABI (jf_compute_dt, jf_stage x 3) with CUDA events
between the calls, so the stage kernel's launch duration is measured live in
the timed region.

Metric: cell-updates per second (cells x RK3 steps / s), whole job (all ranks).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl jf|reference]
                  [--workload tgv256|tgv128|hit384|tgv256_f64] [--extras]

--impl reference times the oracle (FP64 C++ CPU implementation) on a bounded
sample of the same workload on the host cores; it is the reference arm.
Under torchrun (N > 1) each rank advances its own replica of the workload
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (generator, kwargs, dtype)
    "tgv256": ("taylor_green", {"n": 256}, "f32"),
    "tgv128": ("taylor_green", {"n": 128}, "f32"),
    "tgv192": ("taylor_green", {"n": 192}, "f32"),
    "tgv256_f64": ("taylor_green", {"n": 256}, "f64"),
    "tgv128_f64": ("taylor_green", {"n": 128}, "f64"),
    "hit384": ("solenoidal_turbulence", {"n": 384}, "f32"),
    # the paper's ROE setup (flux splitting with the Roe eigensystem, Table 3)
    "tgv256_roe": ("taylor_green", {"n": 256}, "f32"),
    "tgv128_roe": ("taylor_green", {"n": 128}, "f32"),
    "tgv128_roe_f64": ("taylor_green", {"n": 128}, "f64"),
}
# scheme options of a workload (the others run the default HLLC setup)
WORKLOAD_SCHEME = {"tgv256_roe": {"flux": "roe"}, "tgv128_roe": {"flux": "roe"}, "tgv128_roe_f64": {"flux": "roe"}}


def physics_name(case):
    conv = ("ROE setup: Roe flux splitting, WENO5-JS on characteristic fluxes" if case.flux == "roe"
            else "WENO5-JS, HLLC/Einfeldt")
    return f"Navier-Stokes ({conv}, C4 viscous + heat)" if case.viscous else f"Euler ({conv})"


def paper_context(case, dtype):
    """The paper's Table 3 (RTX A6000, JAX): mean wall-clock time per cell and
    step of the same setup and precision; context only (another machine)."""
    table = {("hllc", "f32"): {"64^3": 24.39, "128^3": 25.09, "256^3": 28.36, "384^3": 28.11},
             ("hllc", "f64"): {"64^3": 93.94, "128^3": 92.55, "256^3": 92.76},
             ("roe", "f32"): {"64^3": 302.20, "128^3": 304.55, "256^3": 301.78},
             ("roe", "f64"): {"64^3": 746.78, "128^3": 759.36, "256^3": 760.09}}
    setup = "roe" if case.flux == "roe" else "hllc"
    return {"hardware": "RTX A6000", "setup": setup.upper(), f"ns_per_cell_step_{dtype}": table[(setup, dtype)],
            "source": "Table 3"}


def with_scheme(case, workload):
    for k, v in WORKLOAD_SCHEME.get(workload, {}).items():
        setattr(case, k, v)
    return case

# Algorithmic floating-point operations per cell and per stage launch, as the
# scheme is defined (one evaluation per face), counted by the oracle's
# operation-counting scalar (oracle.count_flops: rhs_per_cell + rk_combine).
FLOPS_PER_CELL_STAGE = {
    (3, True, "hllc"): 3041.0 + 20.0,   # 3D, viscous + heat
    (3, False, "hllc"): 2504.0 + 20.0,  # 3D, inviscid
    (2, True, "hllc"): 1912.0 + 20.0,
    (2, False, "hllc"): 1674.0 + 20.0,
    (1, True, "hllc"): 903.0 + 20.0,
    (1, False, "hllc"): 844.0 + 20.0,
    # ROE setup (flux splitting in characteristic space)
    (3, True, "roe"): 5798.0 + 20.0,
    (3, False, "roe"): 5261.0 + 20.0,
    (2, True, "roe"): 3750.0 + 20.0,
    (2, False, "roe"): 3512.0 + 20.0,
    (1, True, "roe"): 1822.0 + 20.0,
    (1, False, "roe"): 1763.0 + 20.0,
}
# Algorithmic HBM values per cell for the three stages of one RK3 step:
# stage 1 reads Un, writes U1 (10); stages 2 and 3 read U_s and Un and write (15 + 15).
VALUES_PER_CELL_STEP = 40.0
CFL_VALUES_PER_CELL = 5.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="jf", choices=["jf", "reference"])
    p.add_argument("--workload", default="tgv256", choices=sorted(WORKLOADS))
    p.add_argument("--no-extras", action="store_true", help="skip the batched and adjoint measurements")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--variant", type=int, default=-1)
    p.add_argument("--only", choices=["batched", "batched3d", "adjoint", "variants", "learned_flux", "table3"],
                   default=None,
                   help="run only the batched or the adjoint measurement and print it")
    p.add_argument("--adjoint-n", type=int, default=256)
    p.add_argument("--adjoint-steps", type=int, default=400)
    p.add_argument("--adjoint-flow", choices=["kh", "tgv"], default="kh",
                   help="--only adjoint: Kelvin-Helmholtz n^2 (default) or the 3D Taylor-Green vortex n^3")
    return p.parse_args()


def make_case(workload):
    from paper_2203_13760_gb300 import inputs
    gen, kw, dtype = WORKLOADS[workload]
    if gen == "solenoidal_turbulence":
        import torch
        kw = dict(kw, device="cuda" if torch.cuda.is_available() else None)
    return with_scheme(getattr(inputs, gen)(**kw), workload), dtype


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# the files that define the forward stage kernel and its compile flags
STAGE_SOURCES = ("csrc/stage.cuh", "csrc/stage_inst.cuh", "csrc/stage_f32.cu", "csrc/stage_f64.cu",
                 "csrc/stage_f32_gen.cu", "csrc/stage_f64_gen.cu", "csrc/stage_f32_roe.cu",
                 "csrc/stage_f64_roe.cu", "csrc/jf_math.cuh", "csrc/variants.h",
                 "_build.py")


E2E_PASSES = 5  # timed passes of the end-to-end measurement (median reported)


def kernel_sources_sha():
    """Hash of the stage kernel's sources: a recorded ncu traffic figure is
    used only while it matches."""
    h = hashlib.sha256()
    pkg = os.path.join(ROOT, "paper_2203_13760_gb300")
    for name in STAGE_SOURCES:
        with open(os.path.join(pkg, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload, cells):
    """DRAM bytes per stage launch from the committed ncu summary, if it was
    taken on the current kernel sources (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            rec = json.load(f)
    except Exception:
        return None
    if rec.get("sources_sha") != kernel_sources_sha():
        return None
    per_cell = rec.get("stage_bytes_per_cell", {}).get(workload)
    return None if per_cell is None else per_cell * cells


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={device_index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[3:7]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Largest value over the ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, cells_per_rank, steps, max_ms):
    """Whole-job cell-updates/s: every rank advances its own replica (weak
    scaling), the job takes as long as its slowest rank."""
    return world * cells_per_rank * steps / (max_ms * 1e-3)


def cpu_baseline(workload, budget_s=15.0, threads=None):
    """Oracle (FP64 C++, OpenMP over cells) on a bounded sample of the
    workload: the same flow and physics on a 64^3 grid (per-cell work is the
    same as at full size), RK3 steps repeated until ~budget_s of CPU time."""
    import numpy as np

    import oracle
    from paper_2203_13760_gb300 import inputs
    gen, kw, _ = WORKLOADS[workload]
    n = 64
    case = with_scheme(getattr(inputs, gen)(**dict(kw, n=n)), workload)
    c = oracle.config(**case.params())
    cores = oracle.set_threads(threads or os.cpu_count() or 1)
    U = case.U.astype(np.float64)
    steps, t0 = 0, time.perf_counter()
    while True:
        U, _, _ = oracle.run(c, U, 1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or steps >= 400:
            break
    cells = case.cells
    return {"value": cells * steps / el, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{gen} {n}^3 (same physics as {workload}), {steps} CFL RK3 steps in FP64, {el:.1f} s"}


def run_reference(args):
    """Reference arm: the oracle, as it stands, on the host cores."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return 0
    import numpy as np

    import oracle
    from paper_2203_13760_gb300 import inputs
    gen, kw, dtype = WORKLOADS[args.workload]
    n = 48
    case = with_scheme(getattr(inputs, gen)(**dict(kw, n=n)), args.workload)
    c = oracle.config(**case.params())
    cores = oracle.set_threads(os.cpu_count() or 1)
    U = case.U.astype(np.float64)
    for _ in range(args.warmup):
        U, _, _ = oracle.run(c, U, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U, _, _ = oracle.run(c, U, 1)
    el = time.perf_counter() - t0
    value = case.cells * args.steps / el
    line = {
        "impl": "reference", "metric": "cell-updates/s per RK3 step", "value": value, "unit": "cell-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample": f"{gen} {n}^3 per step (bounded sample of the workload)"},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"{gen} {n}^3, same physics, FP64"},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_jf(args):
    import numpy as np
    import torch

    from paper_2203_13760_gb300 import _build
    _build.build()
    from paper_2203_13760_gb300 import jf

    world, rank, local = dist_setup(args)
    case, dtype = make_case(args.workload)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    esize = 4 if dtype == "f32" else 8
    s = jf.Solver.from_case(case, dtype=dtype)
    if args.variant >= 0:
        s.set_variant(args.variant)
    variant = s.variants()[max(args.variant, 0)]
    U0 = torch.from_numpy(case.U.astype(np.float32 if dtype == "f32" else np.float64))
    U = U0.cuda()
    U1 = torch.empty_like(U)
    U2 = torch.empty_like(U)
    dt = s.scalar()
    N = case.cells
    stream = torch.cuda.current_stream()

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        s.compute_dt(U, dt)
        if ev is not None:
            ev[1].record(stream)
        s.stage(U, None, U1, 0.0, 1.0, dt)
        if ev is not None:
            ev[2].record(stream)
        s.stage(U1, U, U2, 0.75, 0.25, dt)
        if ev is not None:
            ev[3].record(stream)
        s.stage(U2, U, U, 1.0 / 3.0, 2.0 / 3.0, dt)
        if ev is not None:
            ev[4].record(stream)

    for _ in range(max(args.warmup, 3)):
        step()
    s.sync()
    K = args.steps
    # the timed region: passes of exactly K steps, each bracketed by a barrier
    # and a device synchronisation, repeated until the passes span >= 1 s (so
    # that the clock record has several samples); the job's value is the
    # median pass
    w0, w1 = _events()
    w0.record(stream)
    for _ in range(3):
        step()
    w1.record(stream)
    torch.cuda.synchronize()
    est_step_ms = w0.elapsed_time(w1) / 3
    passes = int(max(1, min(50, math.ceil(1000.0 / max(K * est_step_ms, 1e-3)))))
    passes = int(max_over_ranks(passes, world))
    events = [[[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(K)] for _ in range(passes)]
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    pass_ms = []
    for r in range(passes):
        barrier(world)
        torch.cuda.synchronize()
        for k in range(K):
            step(events[r][k])
        torch.cuda.synchronize()
        barrier(world)
        pass_ms.append(events[r][0][0].elapsed_time(events[r][-1][4]))
    clk = clocks.stop() if clocks else None
    s.sync()  # raises if a kernel met a non-physical state
    flat = [e for ev in events for e in ev]
    cfl_ms = [e[0].elapsed_time(e[1]) for e in flat]
    stage_ms = [e[i].elapsed_time(e[i + 1]) for e in flat for i in (1, 2, 3)]
    total_ms = max_over_ranks(statistics.median(pass_ms), world)
    ms_per_step = total_ms / K
    value = job_value(world, N, K, total_ms)

    # roofline of the dominant kernel (the stage kernel)
    peaks, peak_kind = measured_peaks()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    stage_avg_s = statistics.mean(stage_ms) * 1e-3
    dim = 3 if case.n[2] > 1 else (2 if case.n[1] > 1 else 1)
    flops = FLOPS_PER_CELL_STAGE.get((dim, bool(case.viscous), "roe" if case.flux == "roe" else "hllc"), None)
    clock_mhz = peaks.get("sm_max_mhz", 2070.0)
    if dtype == "f32":
        peak_tflops = sms * 128 * 2 * clock_mhz * 1e6 / 1e12
    else:
        peak_tflops = 1.25  # nominal GB300 FP64 rate
    achieved_tflops = (flops * N / stage_avg_s / 1e12) if flops else None
    traffic = ncu_traffic(args.workload, N)
    roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": (achieved_tflops / peak_tflops) if achieved_tflops else None, "traffic": traffic,
                "kernel": "stage_kernel", "launch_ms": 1e3 * stage_avg_s,
                "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 (FMA) x {clock_mhz:.0f} MHz"
                if dtype == "f32" else "nominal FP64 rate"}
    # the FMA rate measured on this GPU (jf_fma_peak), beside the derived peak
    try:
        fma_tflops = jf.fma_peak(dtype) / 1e12
    except Exception:  # report the main line even if the microbenchmark fails
        fma_tflops = None
    roofline["measured_fma_peak"] = fma_tflops
    roofline["frac_of_measured_fma"] = (achieved_tflops / fma_tflops) if achieved_tflops and fma_tflops else None
    stage_bytes = (VALUES_PER_CELL_STEP / 3.0) * esize * N
    hbm_gbs = stage_bytes / stage_avg_s / 1e9
    hbm = {"achieved": hbm_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": hbm_gbs / peaks["hbm_gbs"],
           "peak_kind": peak_kind, "step_gbs": (VALUES_PER_CELL_STEP * esize * N) / (ms_per_step * 1e-3) / 1e9,
           "algorithmic_bytes_per_cell_update": VALUES_PER_CELL_STEP * esize}

    # end to end through the public API with host buffers (jf_rk3_step_host):
    # every step uploads its input state from pinned host memory, takes one
    # RK3 step (device CFL) and downloads the result; the library overlaps the
    # copies of the neighbouring states with each step
    Ke = max(3, min(K, 10))
    host_in = [U0.cpu().pin_memory() for _ in range(2)]
    host_out = [torch.empty_like(host_in[0]).pin_memory() for _ in range(Ke)]
    # set-up outside the timed region: the library's buffers and streams, and
    # a first pass of the copies over every host buffer
    s.step_host([host_in[k % 2] for k in range(Ke)], host_out)
    torch.cuda.synchronize()
    barrier(world)
    # E2E_PASSES timed passes of Ke steps; the median pass is reported (the
    # copies share the host's memory and link with whatever else runs on the
    # machine: single passes have run 1.6-2.6x slower than their neighbours)
    e2e_pass_ms = []
    for _ in range(E2E_PASSES):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step_host([host_in[k % 2] for k in range(Ke)], host_out)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_pass_ms.append(e0.elapsed_time(e1))
    s.sync()
    e2e_ms = max_over_ranks(statistics.median(e2e_pass_ms), world)
    e2e = {"value": world * N * Ke / (e2e_ms * 1e-3), "unit": "cell-updates/s",
           "h2d_bytes_per_step": int(host_in[0].numel() * esize),
           "d2h_bytes_per_step": int(host_out[0].numel() * esize),
           "steps_per_pass": Ke, "pass_ms": e2e_pass_ms,
           "call": "jf_rk3_step_host (uploads, steps and downloads overlapped across states); "
                   f"median of {E2E_PASSES} passes"}

    extras = {}
    if not args.no_extras and rank == 0:
        extras = run_extras(args)

    if rank == 0:
        line = {
            "metric": "cell-updates/s per RK3 step", "value": value, "unit": "cell-updates/s", "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": args.workload, "cells": N, "grid": list(case.n), "flow": case.name,
                       "physics": physics_name(case), "integrator": "TVD-RK3, CFL 0.5 on device",
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": "inputs larger than L2 (state %.0f MB)" % (5 * N * esize / 1e6),
                       "variant": variant},
            "roofline": roofline,
            "hbm": hbm,
            "e2e": e2e,
            "gpu_launches": 4 * K * passes,
            "timing": {"passes": passes, "steps_per_pass": K, "pass_ms": pass_ms,
                       "value_from": "median pass (max over ranks)"},
            "clocks": clk,
            "breakdown_ms": {"cfl": statistics.mean(cfl_ms), "stage": statistics.mean(stage_ms)},
            "paper_context": paper_context(case, dtype),
        }
        if extras:
            line["extras"] = extras
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.workload)
            one = cpu_baseline(args.workload, budget_s=5.0, threads=1)
            line["cpu_baseline"]["one_core"] = {"value": one["value"], "cores": one["cores"],
                                                "sample": one["sample"]}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_batched(steps=300, nsim=64, passes=3):
    """64 four-quadrant Riemann problems (sides from {64, 128, 256, 512},
    FP32, CFL steps, 300 steps per pass): one persistent launch per stage over
    all simulations under a captured graph, with the batch tile the autotuner
    picks (cached choice, else timed now), against the same simulations
    advanced one by one through jf_rk3_run (one graph per simulation) and
    through jf_rk3_step.  Each arm: the median of `passes` timed passes."""
    import numpy as np  # noqa: F401
    import torch

    from paper_2203_13760_gb300 import autotune, inputs, jf
    cases = inputs.four_quadrant_batch(nsim=nsim)
    cells = sum(c.cells for c in cases)
    grids = [jf.make_grid(c.n, c.lo, c.hi, c.bc) for c in cases]
    b = jf.Batch(grids, dtype="f32", cfl=0.5)
    fresh = lambda: [torch.tensor(c.U, dtype=torch.float32, device="cuda") for c in cases]  # noqa: E731
    tuned = autotune.apply(b)
    if tuned is None:
        rec = autotune.tune(b, fresh(), steps=3, reps=3)
        tuned, tune_ms = rec["variant"], rec["ms"]
    else:
        tune_ms = "cached"
    variant = b.variants()[tuned]

    U0s = fresh()

    def timed(run, fields):
        """Median of `passes` timed runs on the same field tensors (so that
        no graph is captured again), each from the initial states."""
        out = []
        for _ in range(passes):
            for F, U0 in zip(fields, U0s):
                F.copy_(U0)
            torch.cuda.synchronize()
            e0, e1 = _events()
            e0.record()
            run(fields)
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1) * 1e-3)
        return statistics.median(out), out

    Us = fresh()
    b.step(Us, steps)  # capture + first run
    torch.cuda.synchronize()
    t_batch, batch_passes = timed(lambda F: b.step(F, steps), Us)
    b.sync()
    solvers = [jf.Solver.from_case(c, dtype="f32") for c in cases]
    Vs = fresh()

    def graphs(F):
        for s_, V in zip(solvers, F):
            s_.run(V, steps)

    graphs(Vs)  # capture each simulation's graph
    torch.cuda.synchronize()
    t_graph, _ = timed(graphs, Vs)

    def per_step(F):
        for s_, W in zip(solvers, F):
            for _ in range(steps):
                s_.rk3_step(W)

    Ws = fresh()
    per_step(Ws)
    t_plain, _ = timed(per_step, Ws)
    # the plain arms run each simulation's default tiles; the same bits as
    # the batch (whose last pass started from the initial states) come from
    # the single-grid path with the batch's tiles (row tiles: the same row
    # width and chunk), run once untimed
    m = re.match(r"tile=(\d+)x1 ymarch rows=(\d+) ", variant)
    prefix = f"tile={m[1]}x1 ymarch zchunk={m[2]} " if m else variant.split()[0] + " "
    same = True
    for c, U in zip(cases, Us):
        s_ = jf.Solver.from_case(c, dtype="f32")
        names = s_.variants()
        s_.set_variant(next(i for i, d in enumerate(names) if d.startswith(prefix)))
        W = torch.tensor(c.U, dtype=torch.float32, device="cuda")
        s_.run(W, steps)
        same = same and torch.equal(U, W)
        s_.close()
    # feed_forward: the trajectories of fixed-dt steps (every state kept)
    dts = [0.5 * x for x in b.step(fresh(), 1).tolist()]
    ff_steps = 20
    b.feed_forward(Us, ff_steps, dts)
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    trajs = b.feed_forward(Us, ff_steps, dts)
    e1.record()
    torch.cuda.synchronize()
    t_ff = e0.elapsed_time(e1) * 1e-3
    del trajs
    return {"workload": f"{nsim} four-quadrant Riemann problems, sides {{64,128,256,512}}, FP32, CFL 0.5",
            "cells": cells, "steps": steps, "unit": "cell-updates/s", "passes": passes,
            "timing": "CUDA events, median of the passes; each pass starts from the initial states",
            "variant": variant, "autotune_ms": tune_ms,
            "batched": cells * steps / t_batch, "batched_pass_s": batch_passes,
            "plain_graph_per_sim": cells * steps / t_graph,
            "plain_per_step_calls": cells * steps / t_plain,
            "feed_forward_trajectory": cells * ff_steps / t_ff,
            "feed_forward_note": f"{ff_steps} fixed-dt steps with every state stored (jf_batch_feed_forward)",
            "speedup_vs_graph_per_sim": t_graph / t_batch, "speedup_vs_per_step_calls": t_plain / t_batch,
            "bitwise_equal_to_plain": bool(same), "gpu_launches_batched": 4 * steps}


def run_batched3d(steps=40, nsim=16, passes=3, seed=5):
    """16 Taylor-Green vortices (viscous, FP32, CFL steps) of sides drawn from
    {32, 48, 64, 96, 128} with a seed: one persistent launch per stage over
    the tile columns and z chunks of all simulations (the tile and planes per
    work item the autotuner picks: cached choice, else timed now) under a
    captured graph, against the same simulations advanced one by one through
    jf_rk3_run (one graph per simulation, each with its default variant).
    Median of `passes` passes."""
    import numpy as np
    import torch

    from paper_2203_13760_gb300 import autotune, inputs, jf
    sides = np.random.default_rng(seed).choice([32, 48, 64, 96, 128], size=nsim)
    cases = [inputs.taylor_green(int(n)) for n in sides]
    cells = sum(c.cells for c in cases)
    p = cases[0].params()
    b = jf.Batch([jf.make_grid(c.n, c.lo, c.hi, c.bc) for c in cases], gamma=p["gamma"], R=p["R"], mu=p["mu"],
                 Pr=p["Pr"], dtype="f32", eps=p["eps"], cfl=p["cfl"], viscous=p["viscous"], heat=p["heat"])
    U0s = [torch.tensor(c.U, dtype=torch.float32, device="cuda") for c in cases]
    tuned = autotune.apply(b)
    if tuned is None:
        rec = autotune.tune(b, [u.clone() for u in U0s], steps=3, reps=3)
        tuned, tune_ms = rec["variant"], rec["ms"]
    else:
        tune_ms = "cached"

    def timed(run, fields):
        out = []
        for _ in range(passes):
            for F, U0 in zip(fields, U0s):
                F.copy_(U0)
            torch.cuda.synchronize()
            e0, e1 = _events()
            e0.record()
            run(fields)
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1) * 1e-3)
        return statistics.median(out)

    Us = [u.clone() for u in U0s]
    b.step(Us, steps)  # capture + first run
    torch.cuda.synchronize()
    t_batch = timed(lambda F: b.step(F, steps), Us)
    solvers = [jf.Solver.from_case(c, dtype="f32") for c in cases]
    Vs = [u.clone() for u in U0s]

    def graphs(F):
        for s_, V in zip(solvers, F):
            s_.run(V, steps)

    graphs(Vs)
    torch.cuda.synchronize()
    t_graph = timed(graphs, Vs)
    return {"workload": f"{nsim} Taylor-Green vortices (viscous), sides {sorted(int(x) for x in sides)}, FP32, "
                        "CFL 0.5", "cells": cells, "steps": steps, "unit": "cell-updates/s", "passes": passes,
            "variant": b.variants()[tuned], "autotune_ms": tune_ms, "batched": cells * steps / t_batch,
            "plain_graph_per_sim": cells * steps / t_graph, "speedup_vs_graph_per_sim": t_graph / t_batch}


def run_adjoint(n=256, steps=400, ckpt=20, flow="kh"):
    """Kelvin-Helmholtz 256^2 (Re 1e4), FP32, fixed dt: loss = density L2
    mismatch after 400 steps; gradient w.r.t. the initial state through the
    checkpointed rollout (checkpoints every 20 steps, recompute).  flow="tgv":
    the same protocol on the viscous Taylor-Green vortex n^3 (the 3D adjoint;
    target: the density of the field perturbed off its symmetry planes)."""
    import numpy as np
    import torch

    from paper_2203_13760_gb300 import autograd as jfa
    from paper_2203_13760_gb300 import inputs, jf
    if flow == "tgv":
        case = inputs.taylor_green(n)
        rng = np.random.default_rng(7)
        rho_t = case.U[0] * (1.0 + 1e-3 * rng.standard_normal(case.U[0].shape))
        target = torch.tensor(rho_t, dtype=torch.float32, device="cuda")
        name = f"Taylor-Green {n}^3 Navier-Stokes"
    else:
        case = inputs.kelvin_helmholtz(n)
        target = torch.tensor(inputs.kelvin_helmholtz(n, seed=7).U[0], dtype=torch.float32, device="cuda")
        name = f"Kelvin-Helmholtz {n}^2"
    s = jf.Solver.from_case(case, dtype="f32")
    U0 = torch.tensor(case.U, dtype=torch.float32, device="cuda")
    dt = s.compute_dt(U0)
    # plain forward (one graph of 400 steps)
    V = U0.clone()
    s.run(V, steps, dt)
    torch.cuda.synchronize()
    e0, e1 = _events()
    V = U0.clone()
    e0.record()
    s.run(V, steps, dt)
    e1.record()
    torch.cuda.synchronize()
    t_fwd_graph = e0.elapsed_time(e1) * 1e-3
    # differentiable forward + backward
    X = U0.clone().requires_grad_(True)
    loss = jfa.density_l2(s, jfa.rollout(s, X, steps, dt, ckpt), target)
    loss.backward()
    torch.cuda.synchronize()
    X.grad = None
    e0.record()
    loss = jfa.density_l2(s, jfa.rollout(s, X, steps, dt, ckpt), target)
    e2, e3 = _events()
    e2.record()
    loss.backward()
    e3.record()
    torch.cuda.synchronize()
    t_fwd = e0.elapsed_time(e2) * 1e-3
    t_bwd = e2.elapsed_time(e3) * 1e-3
    s.sync()
    ok = bool(torch.isfinite(X.grad).all().item())
    cells = case.cells
    return {"workload": f"{name}, FP32, {steps} fixed-dt steps, checkpoints every {ckpt}",
            "unit": "cell-updates/s", "forward_graph": cells * steps / t_fwd_graph,
            "forward_differentiable": cells * steps / t_fwd, "backward": cells * steps / t_bwd,
            "backward_over_forward_graph": t_bwd / t_fwd_graph, "grad_finite": ok,
            "backward_ms": 1e3 * t_bwd, "forward_graph_ms": 1e3 * t_fwd_graph}


VARIANT_SCHEMES = {
    "hllc_einfeldt_weno5js_rk3 (default)": {},
    "hll_einfeldt": {"flux": "hll"},
    "rusanov": {"flux": "rusanov"},
    "hllc_davis": {"speeds": "davis"},
    "hllc_toro": {"speeds": "toro"},
    "hllc_weno5z": {"recon": "weno5-z"},
    "hllc_rk2": {"integrator": "rk2"},
    "roe (flux splitting)": {"flux": "roe"},
}


def run_variants(n=256, steps=10):
    """Table 2 scheme variants on the bench flow (TGV n^3, FP32, viscous +
    heat, CFL steps through jf_rk3_step): cell-updates/s per variant.  The
    default row runs the default-scheme kernels, the others the run-time-
    scheme kernels."""
    import torch

    from paper_2203_13760_gb300 import inputs, jf
    case = inputs.taylor_green(n)
    out = {"workload": f"TGV {n}^3 FP32 Navier-Stokes, {steps} CFL steps per variant", "unit": "cell-updates/s"}
    U0 = torch.tensor(case.U, dtype=torch.float32, device="cuda")
    for name, kw in VARIANT_SCHEMES.items():
        s = jf.Solver.from_case(case, dtype="f32", **kw)
        U = U0.clone()
        used = s.scalar()
        for _ in range(2):
            s.rk3_step(U, None, used)
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record()
        for _ in range(steps):
            s.rk3_step(U, None, used)
        e1.record()
        torch.cuda.synchronize()
        s.sync()
        out[name] = case.cells * steps / (e0.elapsed_time(e1) * 1e-3)
        s.close()
    return out


def run_learned_flux(steps=20, warmup=3):
    """Section 7.4 training at the paper's settings (32^2 Rusanov-NN model,
    WENO3-JS / TVD-RK2, batches of 20 windows of 15 steps): time per Adam step
    (forward trajectories with jf_batch_feed_forward, loss, the reverse sweep
    with jf_batch_step_vjp including the parameter gradient), the forward
    alone, and the reference's generation time (128^2 run, 2501 samples)."""
    import time

    import numpy as np
    import torch

    from paper_2203_13760_gb300 import autograd, inputs
    from paper_2203_13760_gb300 import learned_flux as lf
    t0 = time.perf_counter()
    cg = lf.ground_truth(nsamples=2501)
    torch.cuda.synchronize()
    t_ref = time.perf_counter() - t0
    tr = lf.Trainer(cg, inputs.nn_params(seed=0), batch=20, unroll=15, lr=5e-4, n_train=1000, dtype="f32")
    rng = np.random.default_rng(0)
    batches = [rng.choice(tr.starts, 20, replace=False) for _ in range(warmup + steps)]
    for b in batches[:warmup]:
        tr.step(b)
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    torch.cuda.nvtx.range_push("adam_steps")  # lets a profiler select the timed steps
    for b in batches[warmup:]:
        tr.step(b)
    torch.cuda.nvtx.range_pop()
    e1.record()
    torch.cuda.synchronize()
    ms_step = e0.elapsed_time(e1) / steps
    e0.record()
    with torch.no_grad():
        for b in batches[warmup:]:
            autograd.feed_forward(tr.batch, [tr.cg[s] for s in b], tr.unroll, tr.dt)
    e1.record()
    torch.cuda.synchronize()
    ms_fwd = e0.elapsed_time(e1) / steps
    cells = 20 * 15 * cg.shape[-1] * cg.shape[-2]
    return {"workload": "Section 7.4: 32^2 Rusanov-NN, WENO3-JS/TVD-RK2, batch 20 x 15 steps, FP32",
            "ms_per_adam_step": ms_step, "ms_forward_trajectories": ms_fwd,
            "ms_backward_and_loss": ms_step - ms_fwd,
            "forward_cell_updates_per_s": cells / (ms_fwd * 1e-3),
            "reference_seconds": t_ref}


# Table 3 of the paper: ns per cell per RK3 step on the TGV (RTX A6000, JAX; context)
PAPER_TABLE3 = {("hllc", "f32"): {32: 64.41, 64: 24.39, 128: 25.09, 256: 28.36, 384: 28.11},
                ("hllc", "f64"): {32: 98.20, 64: 93.94, 128: 92.55, 256: 92.76},
                ("roe", "f32"): {32: 241.71, 64: 302.20, 128: 304.55, 256: 301.78},
                ("roe", "f64"): {32: 703.40, 64: 746.78, 128: 759.36, 256: 760.09}}


def run_table3(target_s=0.4):
    """The paper's Table 3 workloads on this GPU: TGV n^3 with the HLLC setup
    (WENO5-JS + HLLC) and the ROE setup (flux splitting), FP32 and FP64, CFL
    RK3 steps through jf_rk3_step (Navier-Stokes, the bench physics); ns per
    cell per step next to the paper's."""
    import torch

    from paper_2203_13760_gb300 import inputs, jf
    rows = []
    for (scheme, dtype), paper in PAPER_TABLE3.items():
        sizes = sorted(set(paper) | ({384} if dtype == "f32" else set()))
        for n in sizes:
            case = inputs.taylor_green(n)
            kw = {"flux": "roe"} if scheme == "roe" else {}
            s = jf.Solver.from_case(case, dtype=dtype, **kw)
            t = torch.float32 if dtype == "f32" else torch.float64
            U = torch.tensor(case.U, dtype=t, device="cuda")
            used = s.scalar()
            for _ in range(3):
                s.rk3_step(U, None, used)
            torch.cuda.synchronize()
            e0, e1 = _events()
            e0.record()
            s.rk3_step(U, None, used)
            e1.record()
            torch.cuda.synchronize()
            one = e0.elapsed_time(e1) * 1e-3
            k = max(3, min(200, int(target_s / max(one, 1e-6))))
            e0.record()
            for _ in range(k):
                s.rk3_step(U, None, used)
            e1.record()
            torch.cuda.synchronize()
            s.sync()
            ns = e0.elapsed_time(e1) * 1e6 / (k * case.cells)
            rows.append({"setup": scheme.upper(), "dtype": dtype, "n": n, "steps": k, "ns_per_cell_step": ns,
                         "paper_ns_per_cell_step": paper.get(n),
                         "paper_over_this": (paper[n] / ns) if n in paper else None})
            s.close()
            del U
            torch.cuda.empty_cache()
    return {"workload": "TGV n^3, Navier-Stokes, CFL RK3 steps (paper Table 3 sizes; RTX A6000 numbers as context)",
            "rows": rows}


def run_extras(args):
    """Batched and adjoint forms against the plain per-simulation launch, and
    the scheme variants on the bench flow."""
    out = {}
    try:
        out["batched"] = run_batched()
    except Exception as e:  # report, do not hide the main line
        out["batched"] = {"error": repr(e)}
    try:
        out["adjoint"] = run_adjoint()
    except Exception as e:
        out["adjoint"] = {"error": repr(e)}
    try:
        out["variants"] = run_variants()
    except Exception as e:
        out["variants"] = {"error": repr(e)}
    try:
        out["learned_flux"] = run_learned_flux()
    except Exception as e:
        out["learned_flux"] = {"error": repr(e)}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        import torch

        from paper_2203_13760_gb300 import _build
        _build.build()
        torch.cuda.set_device(0)
        if args.only == "batched":
            out = run_batched()
        elif args.only == "batched3d":
            out = run_batched3d()
        elif args.only == "variants":
            out = run_variants()
        elif args.only == "learned_flux":
            out = run_learned_flux()
        elif args.only == "table3":
            out = run_table3()
        else:
            out = run_adjoint(args.adjoint_n, args.adjoint_steps, flow=args.adjoint_flow)
        print(json.dumps({args.only: out}), flush=True)
        return 0
    return run_jf(args)


if __name__ == "__main__":
    sys.exit(main())
