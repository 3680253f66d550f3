#!/usr/bin/env python3
"""Benchmark of the VLBM time step on one B300 (or N independent replicas, one per GPU).

Workload: the 2D four-quadrant Riemann problem on 4096 x 4096 cells (ideal gas gamma 1.4,
zero-gradient boundaries, CFL 0.5, shock sensor B), seeded synthetic input.  One benchmark
"step" is one vlbm_step call advancing the solver by --substeps time steps (each time step
runs the whole hot path: streaming, moments, EOS, flux, global maxima, link-speed update,
reprojection, sensor, relaxation).  The populations (2.1 GB in FP64) exceed the 126 MB L2, so no
flush is needed between steps.

Reported: FP64 MLUPS (`value`), the FP32-storage variant, the dominant kernel's roofline with its
live CUDA-event duration, the end-to-end number through the C ABI with host buffers, and the
oracle timed on this host's cores.  `--impl reference` times the oracle alone.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--substeps S] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & HBM-roofline fraction: FP64 vs FP32-store fwd; adjoint/fwd time, at stated error"
UNIT = "MLUPS"
# Algorithmic bytes per cell update: every population read once and written once
# (2D: 4 directions x 4 components x 2).
BYTES_PER_CELL = {"fp64": 256, "fp32_store": 128}
# The FP64 step kernel of the two-pass form also reads W, u and Q kept by the maxima pass
# (14 doubles per cell).
FP64_STEP_KERNEL_BYTES = 256 + 112
# Algorithmic FP64 floating-point operations per 2D cell update (ideal gas, shock sensor), FMA
# counted as 2, divide and square root as 1 each: 214 for the whole step.  In the two-pass form
# the maxima pass computes moments, primitives, EOS and flux (and keeps them for the step
# kernel), so the step kernel performs the sensor, filters, beta and the fused
# reprojection/relaxation: 178.
FP64_FLOPS_PER_CELL = 214
FP64_FLOPS_STEP_KERNEL = 178
# Algorithmic bytes of one adjoint step including the recomputation of the forward state (FP64):
# recompute 256 + read the forward state 128 + read lambda 128 + write lambda 128.
ADJ_BYTES_PER_CELL = 640
# FP64 floating-point operations per cell of one adjoint step (the reverse of one time step:
# k_adj_local 237, k_adj_flux 153, k_adj_filter 82; FMA counted as 2), counted by ncu's executed
# DADD/DMUL/DFMA thread instructions on the 1024^2 adjoint workload (profiles/adjoint_kernels_vortex_1024.md).
# The paper gives no operation count for the adjoint; this is the executed arithmetic.
ADJ_FLOPS_PER_CELL = 472
FP64_FMA_PER_CLK_PER_SM = 2  # B300 FP64 unit count per SM (nominal figure, for context)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return {"hbm_gbs": float(d["hbm_gbs"]), "sm_max_mhz": float(d.get("sm_max_mhz", 2032.0)), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0, "source": "fallback"}


def fp64_nominal_tflops(sm_mhz):
    """Dense FP64 rate from unit counts and clock: SMs (of this device) x 2 FP64 FMA/clk x 2 flop x
    f_SM.  Context only; the roofline uses the measured rate."""
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * FP64_FMA_PER_CLK_PER_SM * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during a timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for j, n in enumerate(names):
                    if r[5 + j].strip().lower() in ("active", "1"):
                        reasons.add(n)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# Sources of the step kernels (csrc/), digested by kernels_sha().
KERNEL_SOURCES = ("vlbm_internal.cuh", "vlbm_device.cuh", "vlbm_kernels.cu", "vlbm_roll.cu")


def kernels_sha():
    """Digest of the step-kernel code (the counters in profiles/ are tied to it): the sources with
    comments and blank lines removed, so that a comment edit does not invalidate the counters."""
    import re

    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        src = open(os.path.join(ROOT, "paper_2609_10639_b300", "csrc", name)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in src.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()[:16]


def kernel_traffic(kind):
    """DRAM bytes per cell of the dominant kernel from the committed ncu summary, or None when the
    kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
        entry = d[kind]
    except Exception:
        return None
    digest = kernels_sha()
    if entry.get("kernels_sha") != digest:
        return None
    return float(entry["dram_bytes_per_cell"])


def dist_init():
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world):
    """The maximum of x over the ranks (the slowest replica's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(world, cells, steps, ms):
    """Whole-job throughput of `world` replicas, each advancing `cells` cells by `steps` steps,
    timed by the slowest replica (ms): weak scaling."""
    return world * cells * steps / (ms * 1e-3) / 1e6


def time_path(prob, W0, precision, S, K, W, world, clocks_idx=None, profile=True):
    """Times K vlbm_step(S) calls on device-resident inputs after W untimed ones (with profile, the
    graph chunks carry event-record nodes around every step kernel, read for its mean time)."""
    import torch

    from paper_2609_10639_b300 import vlbm

    s = vlbm.Solver.for_problem(prob, precision=precision)
    s.init(W0)
    for _ in range(W):
        s.step(S)
    s.set_profiling(profile)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(clocks_idx) if clocks_idx is not None else None
    if sampler:
        sampler.__enter__()
    e0.record()
    for _ in range(K):
        done = s.step(S)
        assert done == S
    e1.record()
    torch.cuda.synchronize()
    if sampler:
        sampler.__exit__()
    barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    kms, launches = s.profile()
    s.set_profiling(False)
    lps = s.launches_per_step()
    t, n, c = s.time()
    s.close()
    return {"ms": ms, "kernel_ms_avg": kms / max(launches, 1), "kernel_launches": launches, "launches_per_step": lps,
            "t": t, "n": n, "clocks": sampler.summary() if sampler else None}


def time_e2e(prob, W0_host, precision, S, K, world):
    """Same metric through the C ABI with host buffers: K runs of one vlbm_run_batch call, each
    uploading W0 from pinned host memory, advancing S steps and reading W back into pinned host
    memory (the copies of one run overlap the steps of the next)."""
    import torch

    from paper_2609_10639_b300 import vlbm

    s = vlbm.Solver.for_problem(prob, precision=precision)
    outs = [torch.empty(W0_host.shape, dtype=torch.float64).pin_memory() for _ in range(2)]
    s.run_batch([W0_host] * 2, S, outs=outs)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, done = s.run_batch([W0_host] * K, S, outs=[outs[k & 1] for k in range(K)])
    torch.cuda.synchronize()
    assert done == [S] * K
    dt = max_over_ranks(time.perf_counter() - t0, world)
    s.close()
    nbytes = W0_host.numel() * 8
    return dt, nbytes


def time_adjoint(n_steps, K, world):
    """Reverse-pass time of vlbm_adjoint over the forward time of the same run, on the adjoint
    workload (1024^2 periodic vortex with density perturbation, J = sum g rho(T))."""
    import torch

    from paper_2609_10639_b300 import vlbm, workloads as wl

    prob = wl.VORTEX_ADJOINT_2D
    W0 = torch.from_numpy(wl.vortex_density_2d(prob)).cuda()
    dJ = torch.zeros_like(W0)
    dJ[0] = torch.from_numpy(wl.objective_weight(prob)).cuda()
    s = vlbm.Solver.for_problem(prob)
    s.init(W0)
    s.step(8)  # warm-up of the forward kernels
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.init(W0)
    torch.cuda.synchronize()
    e0.record()
    s.step(n_steps)
    e1.record()
    torch.cuda.synchronize()
    fwd_ms = max_over_ranks(e0.elapsed_time(e1), world)
    s.adjoint(W0, min(n_steps, 2 * K), K, dJ)  # warm-up of the adjoint kernels
    dW0, deos = s.adjoint(W0, n_steps, K, dJ)  # default tape: up to 3/4 of the free HBM
    rev, rec = s.adjoint_timing()
    afwd, taped, tape_bytes = s.adjoint_info()
    rev_ms, rec_ms = max_over_ranks(rev, world), max_over_ranks(rec, world)
    afwd_ms = max_over_ranks(afwd, world)
    s.set_adjoint_tape(0)  # the same run recomputing every segment, for comparison
    s.adjoint(W0, n_steps, K, dJ)
    rev0, rec0 = s.adjoint_timing()
    s.close()
    return {"fwd_ms": fwd_ms, "rev_ms": rev_ms, "rec_ms": rec_ms, "adj_fwd_ms": afwd_ms, "taped_steps": taped,
            "tape_bytes": tape_bytes, "rev_ms_no_tape": max_over_ranks(rev0, world),
            "rec_ms_no_tape": max_over_ranks(rec0, world), "cells": prob.ncells, "steps": n_steps, "K": K}


def oracle_sample(min_seconds=10.0, n=1024, chunk=5, max_steps=None, threads=None):
    """The oracle (as it stands) on a bounded sample of the workload: the same input generator at
    n x n cells, stepped in chunks until min_seconds of CPU work (or max_steps) have run."""
    from oracle import oracle as O
    from paper_2609_10639_b300 import workloads as wl

    p = wl.QUADRANTS_2D.resized(n)
    s = O.OracleSolver.for_problem(p, threads=threads)
    s.init(wl.quadrants_2d(p))
    steps, t0 = 0, time.perf_counter()
    while max_steps is None or steps < max_steps:  # at least one chunk, then until min_seconds
        if steps > 0 and time.perf_counter() - t0 >= min_seconds:
            break
        steps += s.step(chunk if max_steps is None else min(chunk, max_steps - steps))
    dt = time.perf_counter() - t0
    return {"value": p.ncells * steps / dt / 1e6, "unit": UNIT, "cores": s.threads, "kind": "oracle",
            "sample": f"quadrants_2d seed input at {n}x{n}, {steps} FP64 steps from t=0, {dt:.1f} s of CPU work"}


def cpu_baselines():
    """The oracle on all host cores (10 s sample) and on one core (4 s sample)."""
    allc = oracle_sample(min_seconds=10.0)
    one = oracle_sample(min_seconds=4.0, n=512, chunk=2, threads=1)
    allc["one_core"] = {"value": one["value"], "unit": UNIT, "cores": 1, "sample": one["sample"]}
    return allc


def other_workloads(S, K, W, world):
    """FP64 and FP32-storage throughput of the other workloads the library runs: the BZT interface
    with the polytropic van der Waals gas (2048^2), the shock-vortex interaction with its
    pinned-inflow boundary (ideal gas, 800 x 300) and the BZT interface input with the
    non-polytropic gas (c_v(T), FP64 Newton inversion of e -> T; 2048^2)."""
    import torch

    from paper_2609_10639_b300 import workloads as wl

    out = {}
    for prob, make in ((wl.BZT_2D, wl.bzt_interface_2d), (wl.SHOCK_VORTEX_IDEAL, wl.shock_vortex_2d),
                       (wl.BZT_CVT_2D, wl.bzt_interface_2d)):
        W0 = torch.from_numpy(make(prob)).cuda()
        entry = {"grid": [prob.nx, prob.ny]}
        for prec in ("fp64", "fp32_store"):
            # the production graphs for the throughput; a second, profiled run for the step
            # kernel's time (the event-record nodes cost a few us per step, which small grids feel)
            r = time_path(prob, W0, prec, S, K, W, world, profile=False)
            rp = time_path(prob, W0, prec, S, K, W, world)
            entry[prec] = {"value": aggregate_mlups(world, prob.ncells, S * K, r["ms"]), "unit": UNIT,
                           "ms_per_step": r["ms"] / K, "dominant_kernel_ms": rp["kernel_ms_avg"],
                           "value_profiled_run": aggregate_mlups(world, prob.ncells, S * K, rp["ms"])}
        out[prob.name] = entry
    return out


def run_reference(args, n=1024, steps_per_step=8):
    """The reference arm: the oracle timed on the host cores, same metric and workload.  One oracle
    solver is built and warmed up once; each timed step advances it by `steps_per_step` time steps
    of the n x n copy of the workload's input."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    from oracle import oracle as O
    from paper_2609_10639_b300 import workloads as wl

    p = wl.QUADRANTS_2D.resized(n)
    s = O.OracleSolver.for_problem(p)
    s.init(wl.quadrants_2d(p))
    for _ in range(args.warmup):
        s.step(1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        done = s.step(steps_per_step)
        times.append(time.perf_counter() - t0)
        assert done == steps_per_step
    total = sum(times)
    value = p.ncells * steps_per_step * args.steps / total / 1e6
    sample = (f"quadrants_2d seed input at {n}x{n}, one solver, {args.warmup} warm-up steps then {args.steps} x "
              f"{steps_per_step} FP64 steps, {total:.1f} s of CPU work")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.QUADRANTS_2D.name,
                       "sample": f"{n}x{n} copy of the input, {steps_per_step} time steps per step",
                       "parallelism": "host cores (OpenMP)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": s.threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_only(args):
    """One path on an n x n copy of the workload (profiling captures and sweeps)."""
    import torch

    from paper_2609_10639_b300 import workloads as wl

    world, rank, local = dist_init()
    if args.only == "adjoint":
        adj = time_adjoint(args.adjoint_steps, 32, world)
        if rank == 0:
            print(json.dumps({"only": "adjoint", **adj, "reverse_over_forward": adj["rev_ms"] / adj["fwd_ms"],
                              "adjoint_step_over_forward_step": (adj["rev_ms"] - adj["rec_ms"]) / adj["fwd_ms"]}),
                  flush=True)
        return
    prob = wl.QUADRANTS_2D.resized(args.grid) if args.grid else wl.QUADRANTS_2D
    W0 = torch.from_numpy(wl.quadrants_2d(prob)).cuda()
    r = time_path(prob, W0, args.only, args.substeps, args.steps, args.warmup, world)
    if rank == 0:
        mlups = world * prob.ncells * args.substeps * args.steps / (r["ms"] * 1e-3) / 1e6
        kern_gbs = BYTES_PER_CELL[args.only] * prob.ncells / (r["kernel_ms_avg"] * 1e-3) / 1e9
        print(json.dumps({"only": args.only, "workload": prob.name, "grid": [prob.nx, prob.ny], "value": mlups,
                          "unit": UNIT, "ms_per_step": r["ms"] / args.steps, "kernel_ms": r["kernel_ms_avg"],
                          "kernel_alg_gbs": kern_gbs, "t": r["t"], "n": r["n"]}), flush=True)


def run_ours(args):
    import torch

    from paper_2609_10639_b300 import vlbm, workloads as wl  # noqa: F401  (raises if the library is missing)

    world, rank, local = dist_init()
    prob = wl.QUADRANTS_2D
    W0_np = wl.quadrants_2d(prob)
    W0 = torch.from_numpy(W0_np).cuda()
    S, K, Wm = args.substeps, args.steps, args.warmup
    pk = peaks()
    cells = prob.ncells

    fp64_peak = vlbm.measure_fp64_peak(5)  # TFLOP/s, measured on this GPU just before the timed region
    r64 = time_path(prob, W0, "fp64", S, K, Wm, world, clocks_idx=local)
    mlups64 = aggregate_mlups(world, cells, S * K, r64["ms"])
    r32 = time_path(prob, W0, "fp32_store", S, K, Wm, world)
    mlups32 = aggregate_mlups(world, cells, S * K, r32["ms"])

    W0_host = torch.from_numpy(W0_np).pin_memory()
    dt_e2e, nbytes = time_e2e(prob, W0_host, "fp64", S, K, world)
    e2e64 = aggregate_mlups(world, cells, S * K, dt_e2e * 1e3)
    adj = time_adjoint(args.adjoint_steps, 32, world) if args.adjoint_steps > 0 else None
    other = other_workloads(S, min(K, 3), Wm, world) if args.other_workloads else None

    if rank != 0:
        return
    clk = r64["clocks"] or {}
    sm_mhz = clk.get("sm_mhz") or pk["sm_max_mhz"]
    k64_s = r64["kernel_ms_avg"] * 1e-3
    k32_s = r32["kernel_ms_avg"] * 1e-3
    fp64_ach = FP64_FLOPS_STEP_KERNEL * cells / k64_s / 1e12
    fp64_nominal = fp64_nominal_tflops(pk["sm_max_mhz"])
    hbm64 = FP64_STEP_KERNEL_BYTES * cells / k64_s / 1e9
    hbm32 = BYTES_PER_CELL["fp32_store"] * cells / k32_s / 1e9
    t64 = kernel_traffic("fp64_step")
    t32 = kernel_traffic("fp32_store_step")
    cpu = cpu_baselines() if world == 1 else None
    launches = K * (S * r64["launches_per_step"] + 1)
    line = {
        "metric": METRIC, "value": mlups64, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
        "ms_per_step": r64["ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": prob.name, "cells": cells, "grid": [prob.nx, prob.ny], "substeps_per_step": S,
                   "input": f"four-quadrant Riemann problem, seed {wl.quadrant_seed()}, ideal gas 1.4, CFL 0.5",
                   "l2": "inputs larger than L2 (2.1 GB FP64 populations per buffer)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "achieved": fp64_ach, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": fp64_ach / fp64_peak, "traffic": None if t64 is None else t64 * cells,
                     "kernel": "k_roll<double> (FP64 step kernel, column strips, two-pass form)",
                     "kernel_ms": r64["kernel_ms_avg"], "flops_per_cell": FP64_FLOPS_STEP_KERNEL,
                     "peak_source": "measured: vlbm_measure_fp64_peak (chains of dependent FP64 FMAs on every "
                                    "SM, best of 5 launches, just before the timed region)",
                     "peak_nominal": fp64_nominal, "hbm_achieved_gbs": hbm64,
                     "hbm_frac": hbm64 / pk["hbm_gbs"], "hbm_peak_source": pk["source"]},
        "variants": {
            "fp32_store": {"value": mlups32, "unit": UNIT, "dtype": "f32 storage (FP32 math, FP64 maxima)",
                           "ms_per_step": r32["ms"] / K, "speedup_vs_fp64": mlups32 / mlups64,
                           "roofline": {"bound": "hbm", "achieved": hbm32, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                        "frac": hbm32 / pk["hbm_gbs"],
                                        "traffic": None if t32 is None else t32 * cells,
                                        "kernel": "k_roll<float> (FP32-storage step kernel, column strips, look-ahead form: the whole step in one pass)",
                                        "kernel_ms": r32["kernel_ms_avg"], "peak_source": pk["source"],
                                        "bytes_per_cell": BYTES_PER_CELL["fp32_store"]}},
            "other_workloads": other,
            "adjoint": None if adj is None else {
                "workload": "vortex_adjoint_2d_1024 (J = sum g rho(T), checkpoints every 32 steps)",
                "value": world * adj["cells"] * adj["steps"] / (adj["rev_ms"] * 1e-3) / 1e6, "unit": UNIT,
                "dtype": "f64", "steps": adj["steps"], "forward_ms": adj["fwd_ms"], "reverse_ms": adj["rev_ms"],
                "recompute_ms": adj["rec_ms"],
                "reverse_over_forward": adj["rev_ms"] / adj["fwd_ms"],
                "adjoint_step_over_forward_step": (adj["rev_ms"] - adj["rec_ms"]) / adj["fwd_ms"],
                "tape": {"taped_steps": adj["taped_steps"], "bytes": adj["tape_bytes"],
                         "note": "the forward pass keeps the last segments' states (with their sensor planes, "
                                 "and W, u, Q where memory is left) in HBM, up to 3/4 of the free memory, so the "
                                 "reverse pass recomputes only the other segments"},
                "adjoint_forward_pass_ms": adj["adj_fwd_ms"],
                "whole_call_over_forward": (adj["adj_fwd_ms"] + adj["rev_ms"]) / adj["fwd_ms"],
                "without_tape": {"reverse_ms": adj["rev_ms_no_tape"], "recompute_ms": adj["rec_ms_no_tape"],
                                 "reverse_over_forward": adj["rev_ms_no_tape"] / adj["fwd_ms"]},
                "roofline": {"bound": "alu", "unit": "TFLOP/s", "peak": fp64_peak,
                             "achieved": ADJ_FLOPS_PER_CELL * adj["cells"] * adj["steps"]
                                         / ((adj["rev_ms"] - adj["rec_ms"]) * 1e-3) / 1e12,
                             "frac": ADJ_FLOPS_PER_CELL * adj["cells"] * adj["steps"]
                                     / ((adj["rev_ms"] - adj["rec_ms"]) * 1e-3) / 1e12 / fp64_peak,
                             "flops_per_cell": ADJ_FLOPS_PER_CELL,
                             "kernels": "the adjoint-step kernels (k_adj_local, k_adj_flux, k_adj_filter and "
                                        "the folds) over the reverse pass minus its segment recomputation",
                             "note": "every adjoint kernel is FP64-pipe bound (ncu: "
                                     "profiles/adjoint_kernels_vortex_1024.md); a step taped in a lean slot "
                                     "also evaluates W, u, Q (k_adj_fields, not counted in flops_per_cell)",
                             "hbm_achieved_gbs": ADJ_BYTES_PER_CELL * adj["cells"] * adj["steps"] / (adj["rev_ms"] * 1e-3) / 1e9,
                             "hbm_frac": ADJ_BYTES_PER_CELL * adj["cells"] * adj["steps"] / (adj["rev_ms"] * 1e-3) / 1e9 / pk["hbm_gbs"],
                             "hbm_bytes_per_cell": ADJ_BYTES_PER_CELL}},
        },
        "cpu_baseline": cpu,
        "e2e": {"value": e2e64, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
        "gpu_launches": launches,
        "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"), "reasons": clk.get("reasons", []),
                   "samples": clk.get("samples", 0)},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--substeps", type=int, default=32)
    ap.add_argument("--adjoint-steps", type=int, default=1000, help="steps of the adjoint measurement (0: skip)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--other-workloads", type=int, default=1, help="also time the shock-vortex and non-polytropic "
                                                                       "workloads (0: skip)")
    ap.add_argument("--only", choices=list(BYTES_PER_CELL) + ["adjoint"],
                    help="time one path only (profiling, sweeps); adjoint: the adjoint measurement alone")
    ap.add_argument("--grid", type=int, default=0, help="with --only: n x n copy of the workload")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.only:
        run_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
