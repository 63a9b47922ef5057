#!/usr/bin/env python
"""Benchmark of the D3Q39 13-moment DDF lattice Boltzmann step (MLUPS) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload box256|box384|box128|box2d|naca|sod|poly|serve]
                    [--precision fp64|mixed] [--sections precision,serving,airfoil,root_finders,prandtl|none]

A step is one full time step (collide + stream with the mask rules) over the whole
lattice.  Inputs are synthetic and seeded (paper_1910_13515_gb300.inputs).  The default
line is the 3-D periodic 256^3 box in FP64 (rms Ma 0.8); the same line carries the other
parts of the metric: the precision form on the 256^3 and 384^3 boxes against the FP64
path, a serving run (Poisson request stream, p50/p99 time-to-solution, aggregate MLUPS
against serial stepping), the 2048x1024 NACA0012 airfoil (early window and developed
flow), the other root finders and stopping tolerances on the 256^3 box, and the
Prandtl-number adjustment (Pr = 0.71) on the same box.  For N > 1 (torchrun, one process
per GPU) every rank runs its own replica of the
workload (weak scaling; the step has no exchange between replicas) and the extra sections
are skipped.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3Q39 DDF MLUPS & HBM-roofline fraction, FP64 vs mixed; serving p50/p99 ms"

WORKLOADS = {
    "naca": "NACA0012 supersonic flow, 2048x1024x1 cells, C=400, Ma=1.5, Re=1e4, bounce-back "
            "airfoil, freestream left/top/bottom, outflow right, alpha(eps) on",
    "box256": "3-D periodic box 256^3, solenoidal velocity rms Ma=0.8, +-5% rho/T noise, "
              "seed 0, tau=0.55, alpha(eps) on",
    "box384": "3-D periodic box 384^3, solenoidal velocity rms Ma=0.8, +-5% rho/T noise, "
              "seed 0, tau=0.55, alpha(eps) on",
    "box128": "3-D periodic box 128^3 (profiling size), solenoidal velocity rms Ma=0.8, "
              "+-5% rho/T noise, seed 0, tau=0.55, alpha(eps) on",
    "box2d": "quasi-2-D periodic box 2048x1024x1, solenoidal velocity scaled to rms Ma=0.8 with "
             "u_z then set to 0 (z-mirror symmetric), +-5% rho/T noise, seed 0, tau=0.55, "
             "alpha(eps) on",
    "sod": "Sod tube 400x1x1, outflow ends, tau=0.5 with alpha(eps)",
    "poly": "polynomial-equilibrium comparison model (D3Q39 DDF-BGK, 4th-order Hermite "
            "equilibrium), periodic NxNx1 (default 2048, the paper's comparison size), subsonic solenoidal flow rms Ma=0.3 at T=2/3, "
            "+-1% rho/T noise, tau=0.6, plain BGK",
    "serve": "serving form: Poisson stream of 64 seeded requests (Riemann tubes 200-4000 cells, "
             "2-D shear layers 128^2-1024^2, 200-2000 steps), admitted into a 4 GiB budget",
}

# FP64 arithmetic of one fluid-cell update as executed by the step kernel, from ncu
# instruction counts (2 flops per DFMA, 1 per DADD/DMUL) on two workloads with different
# Newton work: A + B * (Newton updates per cell) [+ C * (share of solves with a single-
# precision start)].  See profiles/.
FP64_FLOPS_MODEL = {
    # the 128^3 box at rms Ma 0.8 (3.97 updates per cell: 10509 flops per cell) and 0.3
    # (3.21: 8619)
    "fp64": (691.0, 2472.0),
    # the precision form (single-precision start, then FP32-direction Newton steps): its
    # per-cell part and per-update cost from the form without the start (3.99 updates per
    # cell: 4722 flops per cell), and C, the full FP64 evaluation that a solve after a start
    # takes in place of the cached one, from the 128^3 box at rms Ma 0.8 (2.003 updates, every
    # solve started: 3401) and 0.3 (1.982: 3375)
    "mixed": (542.0, 1051.0, 752.0),
    # the nine-constraint (z-mirror) solve of lattices one cell thick in z: the 2048x1024
    # airfoil at 0.018 updates per cell (686 flops per cell) and the quasi-2-D 2048x1024 box
    # at 3.26 (5129)
    "fp64_2d": (661.0, 1369.0),
    # FP64 storage with the single-precision Newton direction (root finder 2): the FP64 path's
    # per-cell part and the 128^3 box's count (4869 flops per cell at 3.99 updates per cell)
    "fp64_fp32dir": (691.0, 1047.0),
    # root finder 3 (2 after a single-precision start): as root finder 2, with C from the
    # 128^3 box at rms Ma 0.8 (2.003 updates, every solve started: 3552 flops per cell) and
    # 0.3 (1.982: 3526)
    "fp64_fp32start": (691.0, 1047.0, 761.0)}
# DRAM bytes (read + write) per launch of the step kernel from ncu, per workload and
# precision, with the hash of the step kernel's code they were captured with; reported as
# null once that code differs (profiles/ has the captures).  The 256^3 and 384^3 figures are
# the 128^3 captures scaled by the cell count (x 8, x 27; the same per-cell work, all far
# beyond L2).
NCU_TRAFFIC = {"kernel_hash": "98f81eefb40860d3",
               "gb_per_launch": {"box128/fp64": 4.705, "box256/fp64": 37.64,
                                 "box128/mixed": 3.069, "box256/mixed": 24.55,
                                 "box384/mixed": 82.86}}
# The sources the step kernels and their launches are built from (the serving-form kernels
# in batch.cuh are not among them).
KERNEL_SOURCES = ("cell.cuh", "d3q39.cuh", "d3q39_gen.cuh", "expd.cuh", "kernels.cuh",
                  "lbm39.cu")
# The same for the polynomial comparison model's step kernel, and its ncu DRAM bytes per
# launch (per lattice side n of the n x n x 1 workload; null once the code differs).
POLY_SOURCES = ("cell.cuh", "d3q39.cuh", "d3q39_gen.cuh", "expd.cuh", "kernels.cuh",
                "poly_eq.cuh", "poly.cu")
POLY_NCU_TRAFFIC = {"kernel_hash": "02dc9070eca147c2",
                    # 2048: the 1024 capture scaled by the cell count (both exceed L2)
                    "gb_per_launch": {"1024": 1.272, "2048": 5.087}}


def source_code_text(text: str) -> str:
    """C/CUDA source with its comments removed and its whitespace runs made single
    spaces: the text a compiler acts on, so that comment edits keep the hash."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return " ".join(text.split())


def kernel_source_hash(sources=KERNEL_SOURCES) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_1910_13515_gb300", "csrc", f)) as fh:
            h.update(source_code_text(fh.read()).encode())
        h.update(b"\0")
    return h.hexdigest()[:16]
# FP64 flops of one cell update of the polynomial comparison model, counted from its source
# (2 per FMA, identical subexpressions once): moments 120, sum g 38, rho/u/T 21, cell
# coefficients 35, shell coefficients 70, rest velocity 7, xi.u 32, 19 (xi, -xi) pairs x 20.
POLY_FLOPS_PER_UPDATE = 703
# populations read + written, and the per-cell solver state (lam and F: 52 FP64) read + written
BYTES_PER_UPDATE = {"fp64": 78 * 8 * 2 + 52 * 8 * 2, "mixed": 78 * 4 * 2 + 52 * 8 * 2}


def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0  # fallback figure of the profiling recipe


HBM_PEAK_GBS = _hbm_peak()


def make_setup(name: str, mach: float = 0.8):
    from paper_1910_13515_gb300 import inputs
    if name == "naca":
        return inputs.naca()
    if name == "box256":
        return inputs.box(n=256, seed=0, mach_rms=mach)
    if name == "box384":
        return inputs.box(n=384, seed=0, mach_rms=mach)
    if name == "box128":
        return inputs.box(n=128, seed=0, mach_rms=mach)
    if name == "box2d":
        s = inputs.box(seed=0, mach_rms=mach, shape=(1, 1024, 2048))
        s.u[2] = 0.0  # in-plane flow: z-mirror symmetric
        return s
    if name == "sod":
        return inputs.sod(400)
    raise ValueError(name)


def workload_text(args) -> str:
    text = WORKLOADS[args.workload]
    if args.workload.startswith("box") and args.mach != 0.8:
        text = text.replace("rms Ma=0.8", f"rms Ma={args.mach:g}")
    if args.workload == "poly":
        n = getattr(args, "poly_n", 2048)
        text = text.replace("periodic NxNx1 (default 2048, the paper's comparison size)",
                            f"periodic {n}x{n}x1" + (" (the paper's comparison size)"
                                                      if n == 2048 else ""))
    return text


def crop_setup(s, name: str):
    """Bounded sample of a workload for the CPU oracle: a window of the same lattice
    (same masks and fields), periodic at the window edges."""
    import copy

    import numpy as np
    if name == "naca":
        win = (slice(0, 1), slice(384, 640), slice(448, 960))   # around the airfoil
    elif name.startswith("box"):
        win = (slice(0, 48), slice(0, 48), slice(0, 48))
    else:
        return s, "the whole lattice"

    def cut(a):
        a3 = a.reshape(-1, s.nz, s.ny, s.nx)[(slice(None),) + win]
        return np.ascontiguousarray(a3.reshape(a3.shape[0], -1))

    c = copy.copy(s)
    c.nz, c.ny, c.nx = (w.stop - w.start for w in win)
    c.periodic = (1, 1, 1)
    c.mask = cut(s.mask)[0]
    c.rho, c.u, c.T = cut(s.rho)[0], cut(s.u), cut(s.T)[0]
    return c, f"{c.nx}x{c.ny}x{c.nz} window of the same lattice (periodic at the window edges)"


def oracle_mlups(s, steps: int, budget_s: float = None):
    """Time the FP64 CPU oracle (as it stands) on setup s; returns (MLUPS, steps, threads)."""
    from oracle import oracle39 as o
    cfg = o.Config(nx=s.nx, ny=s.ny, nz=s.nz, periodic=s.periodic, gamma=s.gamma, tau=s.tau,
                   kn_sensor=s.kn_sensor, rho_inf=s.rho_inf, u_inf=s.u_inf, T_inf=s.T_inf)
    st = o.init(cfg, s.mask, s.rho, s.u, s.T)
    done = 0
    t0 = time.perf_counter()
    while done < steps:
        o.step(st, 1)
        done += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return s.ncells * done / dt / 1e6, done, threads, dt


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = sorted(float(r[1]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


def poly_window(s, n: int = 128):
    """n x n window of a quasi-2-D setup (periodic at the window edges): the polynomial
    model's bounded CPU sample."""
    import copy

    import numpy as np
    c = copy.copy(s)
    sel = (np.arange(n)[:, None] * s.nx + np.arange(n)[None, :]).reshape(-1)
    c.nx, c.ny, c.nz = n, n, 1
    c.rho, c.u, c.T = s.rho[sel], np.ascontiguousarray(s.u[:, sel]), s.T[sel]
    c.mask = s.mask[sel]
    return c, f"{n}x{n}x1 window of the same lattice (periodic at the window edges)"


def poly_oracle_steps(c, warmup: int, steps: int, budget_s: float = None):
    """Time the polynomial model's oracle (numpy, as it stands) on setup c."""
    from oracle import poly39
    cfg = poly39.Config(nx=c.nx, ny=c.ny, nz=c.nz, gamma=c.gamma, tau=c.tau)
    st = poly39.init(cfg, c.rho, c.u, c.T)
    poly39.step(st, warmup)
    done = 0
    t0 = time.perf_counter()
    while done < steps:
        poly39.step(st, 1)
        done += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return c.ncells * done / dt / 1e6, done, dt


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle as it stands, on the host cores, each step a
    bounded sample (a window) of the same workload."""
    if rank != 0:
        return
    if args.workload == "poly":
        from paper_1910_13515_gb300 import inputs
        c, desc = poly_window(inputs.subsonic_box(args.poly_n, args.poly_n, 1, seed=0),
                              min(128, args.poly_n))
        v, done, dt = poly_oracle_steps(c, args.warmup, args.steps)
        line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "MLUPS",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload_text(args) + f" [oracle on a {desc}]",
                           "cells": c.ncells},
                "cpu_baseline": {"value": round(v, 4), "unit": "MLUPS", "cores": 1,
                                 "kind": "oracle", "sample": desc},
                "e2e": {"value": round(v, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    s = make_setup(args.workload, args.mach)
    c, desc = crop_setup(s, args.workload)
    from oracle import oracle39 as o
    cfg = o.Config(nx=c.nx, ny=c.ny, nz=c.nz, periodic=c.periodic, gamma=c.gamma, tau=c.tau,
                   kn_sensor=c.kn_sensor, rho_inf=c.rho_inf, u_inf=c.u_inf, T_inf=c.T_inf)
    st = o.init(cfg, c.mask, c.rho, c.u, c.T)
    o.step(st, args.warmup)
    t0 = time.perf_counter()
    o.step(st, args.steps)
    dt = time.perf_counter() - t0
    v = c.ncells * args.steps / dt / 1e6
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_text(args) + f" [oracle on a {desc}]",
                       "cells": c.ncells},
            "cpu_baseline": {"value": round(v, 4), "unit": "MLUPS", "cores": threads,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": round(v, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def reduce_over_ranks(elapsed_s: float, units: float, dist=None, device=None):
    """Whole-job timing of weak-scaled replicas: the slowest rank's time and the units all
    ranks processed (each rank runs its own lattice; no data-path collective)."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return elapsed_s, units
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def serving_section(args, local, n_requests: int, rate_hz: float, seed: int = 0):
    """The serving form on a Poisson stream of n_requests seeded requests: aggregate MLUPS
    over the whole stream (all cells x steps of all requests / wall time from first arrival
    to last result) and p50/p99 time-to-solution (arrival to result read).  Baseline: the
    same requests run one after another through plain lbm39_step (no packing), each with its
    own init and read-out, as a served request has -- all of them, so that the baseline has
    the stream's mix of lattice sizes (a sample without the large shear layers would run
    the small, launch-bound lattices only)."""
    import torch

    from paper_1910_13515_gb300 import inputs
    from paper_1910_13515_gb300.lattice import Lattice
    from paper_1910_13515_gb300.serve import GpuBackend, Scheduler

    prec = 0 if args.precision == "fp64" else 1
    reqs = inputs.serving_requests(n_requests, seed=seed, rate_hz=rate_hz)
    be = GpuBackend(precision=prec, max_lattices=64, max_cells=1 << 25,
                    graph_steps=8, device=f"cuda:{local}")
    warm = inputs.serving_requests(4, seed=1000 + seed, rate_hz=1e6, shear_sizes=(128,),
                                   riemann_range=(200, 400), steps_range=(16, 24))
    Scheduler(be, 4 << 30, 64, chunk_steps=64).run(warm)
    with ClockSampler(local) as clk:
        rep = Scheduler(be, 4 << 30, 64, chunk_steps=64).run(reqs)
    clocks = clk.summary()
    be.close()
    sample = reqs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cs = 0
    for r in sample:
        L = Lattice.from_setup(r.setup, precision=prec, device=f"cuda:{local}")
        L.step(r.setup.steps)
        L.read_numpy()
        cs += r.setup.ncells * r.setup.steps
        L.close()
    serial = cs / (time.perf_counter() - t0) / 1e6
    return {"requests": len(reqs), "arrival_rate_hz": rate_hz, "budget_gib": 4,
            "cell_steps": rep.cell_steps, "max_resident": rep.max_resident,
            "rounds": rep.rounds, "requests_with_fallback_cells": len(rep.failed),
            "p50_ms": round(rep.p50_ms, 2), "p99_ms": round(rep.p99_ms, 2),
            "aggregate_mlups": round(rep.mlups, 3), "serial_mlups": round(serial, 3),
            "speedup_vs_serial": round(rep.mlups / serial, 3),
            "serial_sample": f"all {len(sample)} requests, one at a time",
            "wall_s": round(rep.wall_s, 2), "clocks": clocks}


def run_serve(args, rank, world, local):
    """The serving form as its own line: value = aggregate MLUPS of the request stream."""
    import torch
    torch.cuda.set_device(local)
    sec = serving_section(args, local, 64, args.serve_rate, seed=rank)
    if rank == 0:
        prec = 0 if args.precision == "fp64" else 1
        line = {"metric": METRIC, "value": sec["aggregate_mlups"], "unit": "MLUPS",
                "n_gpus": world, "steps": sec["cell_steps"], "warmup": 4,
                "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if prec == 0 else "f32-storage/f64-solve",
                "data": "synthetic",
                "config": {"workload": WORKLOADS["serve"], "requests": sec["requests"],
                           "cell_steps": sec["cell_steps"], "budget_gib": 4,
                           "max_resident": sec["max_resident"], "rounds": sec["rounds"],
                           "arrival_rate_hz": args.serve_rate},
                "serving": {k: v for k, v in sec.items() if k != "clocks"},
                "clocks": sec["clocks"], "gpu_launches": None}
        print(json.dumps(line), flush=True)


def run_poly(args, rank, world, local):
    """The polynomial-equilibrium comparison model on the paper's comparison size: value =
    MLUPS of lbm39_poly_step (device-timed), roofline against the FP64 pipe (the binding one at
    703 flops and 1248 bytes per update), e2e through PolyLattice with host buffers."""
    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_1910_13515_gb300 import inputs
    from paper_1910_13515_gb300 import lbm39 as C
    from paper_1910_13515_gb300.lattice import PolyLattice

    dev = f"cuda:{local}"
    n = args.poly_n
    s = inputs.subsonic_box(n, n, 1, seed=0)
    N = s.ncells
    L = PolyLattice(s.nx, s.ny, s.nz, gamma=s.gamma, tau=s.tau, device=dev)
    L.init(s.rho, s.u, s.T)
    c0 = L.conserved()
    L.step(args.warmup)
    stream = L.stream
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        evs[0].record(stream)
        for k in range(args.steps):
            L.step(1)
            evs[k + 1].record(stream)
        torch.cuda.synchronize()
        barrier()
    clocks = clk.summary()
    per_step = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    elapsed_s, units = reduce_over_ranks(evs[0].elapsed_time(evs[-1]) * 1e-3,
                                         float(N * args.steps), dist, dev)
    value = units / elapsed_s / 1e6
    c1 = L.conserved()
    step_ms = float(np.mean(per_step))
    scratch = torch.empty(1 << 21, dtype=torch.float64, device=dev)
    rc, peak_tf = C.lbm39_selftest_dfma(scratch.data_ptr(), scratch.numel() * 8,
                                        stream.cuda_stream)
    C.check(rc, "lbm39_selftest_dfma")
    achieved_tf = POLY_FLOPS_PER_UPDATE * N / (step_ms * 1e-3) / 1e12
    bytes_upd = 78 * 8 * 2
    hbm_gbs = bytes_upd * N / (step_ms * 1e-3) / 1e9
    traffic = None
    if POLY_NCU_TRAFFIC["kernel_hash"] == kernel_source_hash(POLY_SOURCES):
        traffic = POLY_NCU_TRAFFIC["gb_per_launch"].get(str(n))
    roofline = {"bound": "alu", "achieved": round(achieved_tf, 4), "peak": round(peak_tf, 4),
                "unit": "TFLOP/s", "frac": round(achieved_tf / peak_tf, 4),
                "traffic": round(traffic * 1e9) if traffic else None,
                "peak_source": "FP64 FMA throughput measured in this run by lbm39_selftest_dfma "
                               "(of measured)",
                "flops_per_cell_update": POLY_FLOPS_PER_UPDATE,
                "flops_source": "counted from the kernel source, not from ncu",
                "hbm": {"achieved_gbs": round(hbm_gbs, 1), "peak_gbs": HBM_PEAK_GBS,
                        "frac": round(hbm_gbs / HBM_PEAK_GBS, 4), "bytes_per_update": bytes_upd}}

    # end to end through PolyLattice: fields uploaded from pinned host memory, then every step
    # a step, a read-out and its copy into pinned host memory
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64)).pin_memory()
        h_rho, h_u, h_T = pin(s.rho), pin(s.u), pin(s.T)
        h_out = torch.empty((6, N), dtype=torch.float64).pin_memory()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L.init(h_rho.to(dev, non_blocking=True), h_u.to(dev, non_blocking=True),
               h_T.to(dev, non_blocking=True))
        for _ in range(args.steps):
            L.step(1)
            r, u, T, p = L.read()
            h_out[0].copy_(r, non_blocking=True)
            h_out[1:4].copy_(u, non_blocking=True)
            h_out[4].copy_(T, non_blocking=True)
            h_out[5].copy_(p, non_blocking=True)
            torch.cuda.current_stream(dev).synchronize()
        dt, units_e2e = reduce_over_ranks(time.perf_counter() - t0, float(N * args.steps),
                                          dist, dev)
        e2e = {"value": round(units_e2e / dt / 1e6, 3), "unit": "MLUPS",
               "h2d_bytes_per_step": int(5 * 8 * N / args.steps), "d2h_bytes_per_step": 6 * 8 * N,
               "steps": args.steps, "includes": "upload of rho,u,T + lbm39_poly_init once, per "
                                               "step lbm39_poly_step(1), lbm39_poly_read and the "
                                               "copy of rho,u,T,p to pinned host memory"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        c, desc = poly_window(s)
        v, done, dt = poly_oracle_steps(c, 0, 10 ** 6, budget_s=args.cpu_budget_s)
        cpu = {"value": round(v, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
               "sample": f"{desc}: {done} numpy oracle steps in {dt:.1f} s"}

    if rank == 0:
        drift = (np.abs(c1 - c0) / np.array([c0[0]] * 4 + [c0[4]])).tolist()
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(elapsed_s * 1e3 / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_text(args), "model": "polynomial", "cells": N,
                       "conservation_drift_rel_mass_mom_xyz_energy":
                           [float("%.3e" % v) for v in drift],
                       "l2": "inputs larger than L2 (%.2f GB of populations)" % (
                           bytes_upd / 2 * N / 1e9),
                       "parallelism": "replicas" if world > 1 else "1 GPU"},
            "clocks": clocks, "roofline": roofline, "e2e": e2e,
            "gpu_launches": args.steps, "cpu_baseline": cpu,
            "kernel_hash": kernel_source_hash(POLY_SOURCES),
        }
        print(json.dumps(line), flush=True)
    L.close()
    if world > 1:
        dist.destroy_process_group()


def timed_steps(L, steps: int, local: int, barrier=lambda: None):
    """K steps of lattice L, each bracketed by CUDA events on the lattice's stream, with the
    clocks sampled meanwhile: (per-step ms list, total ms, clock summary)."""
    import torch
    stream = L.stream
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        evs[0].record(stream)
        for k in range(steps):
            L.step(1)
            evs[k + 1].record(stream)
        torch.cuda.synchronize()
        barrier()
    clocks = clk.summary()
    per_step = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
    return per_step, evs[0].elapsed_time(evs[-1]), clocks


def counter_shares(st0, st1, cell_steps: int) -> dict:
    """Newton-update and alpha-branch shares of the cell updates between two stats reads."""
    hist = [st1.newton_hist[k] - st0.newton_hist[k] for k in range(32)]
    return {"newton_updates_per_cell": round((st1.newton_updates - st0.newton_updates)
                                             / cell_steps, 4),
            "newton_updates_share_0_1_2_3_4plus":
                [round(h / cell_steps, 4) for h in hist[:4]] + [round(sum(hist[4:]) / cell_steps, 4)],
            "alpha_branch_share": [round((st1.eps_hist[k] - st0.eps_hist[k]) / cell_steps, 4)
                                   for k in range(4)],
            "fallback_share": round((st1.failed_cells - st0.failed_cells) / cell_steps, 6),
            "start32_steps_per_cell": round((st1.start32_updates - st0.start32_updates)
                                            / cell_steps, 4),
            "start32_solve_share": round((st1.start32_solves - st0.start32_solves)
                                         / cell_steps, 4)}


def l1_rel(a, b, fl):
    """L1 differences of (rho, u, T) fields a against b over the fluid cells, each relative to
    the L1 norm of b (u: of |u|)."""
    import numpy as np
    (ra, ua, Ta), (rb, ub, Tb) = a[:3], b[:3]
    return [float(np.abs(ra[fl] - rb[fl]).mean() / np.abs(rb[fl]).mean()),
            float(np.abs(ua[:, fl] - ub[:, fl]).mean() / np.sqrt((ub[:, fl] ** 2).sum(0)).mean()),
            float(np.abs(Ta[fl] - Tb[fl]).mean() / np.abs(Tb[fl]).mean())]


def drift_rel(c0, c1):
    """Relative change of the conserved sums (mass, momentum x/y/z relative to the mass,
    energy)."""
    import numpy as np
    c0, c1 = np.array(c0), np.array(c1)
    return (np.abs(c1 - c0) / np.array([abs(c0[0])] * 4 + [abs(c0[4])])).tolist()


def precision_form_section(args, local, s256, fp64_256):
    """The precision form (FP32 deviation storage, FP32 collision, FP64 moments and solve) on
    the 256^3 and 384^3 boxes, against the FP64 path on the same input after the same steps
    (the FP64 path is parity-checked against the FP64 oracle): MLUPS, speed-up, L1 error in
    rho/u/T, conservation drift.  fp64_256: (fields, MLUPS) of the FP64 256^3 run."""
    import torch

    from paper_1910_13515_gb300 import lbm39 as C
    from paper_1910_13515_gb300.lattice import Lattice
    dev = f"cuda:{local}"
    out = {}
    nsteps = args.warmup + args.steps
    for n in (256, 384):
        s = s256 if n == 256 else make_setup("box384", args.mach)
        fl = s.mask == 0
        if n == 256:
            ref, ref_mlups = fp64_256
        else:
            Lf = Lattice.from_setup(s, precision=C.LBM39_FP64, device=dev)
            Lf.step(args.warmup)
            _, ms, _ = timed_steps(Lf, args.steps, local)
            ref_mlups = s.ncells * args.steps / (ms * 1e-3) / 1e6
            ref = Lf.read_numpy()
            Lf.close()
            del Lf
            torch.cuda.empty_cache()
        Lm = Lattice.from_setup(s, precision=C.LBM39_MIXED, device=dev)
        c0 = Lm.stats().conserved
        Lm.step(args.warmup)
        st0 = Lm.stats()
        per_step, ms, clocks = timed_steps(Lm, args.steps, local)
        st1 = Lm.stats()
        mlups = s.ncells * args.steps / (ms * 1e-3) / 1e6
        state = Lm.read_numpy()
        Lm.close()
        del Lm
        torch.cuda.empty_cache()
        drift = drift_rel(c0, st1.conserved)
        sec = {"cells": s.ncells, "mlups": round(mlups, 3), "fp64_mlups": round(ref_mlups, 3),
               "speedup_vs_fp64": round(mlups / ref_mlups, 3),
               "compared_after_steps": nsteps,
               "l1_rel_vs_fp64_rho_u_T": [float("%.3e" % v) for v in l1_rel(state, ref, fl)],
               "conservation_drift_rel_mass_mom_xyz_energy": [float("%.3e" % v) for v in drift],
               "conservation_drift_per_1000_steps": [float("%.3e" % (v * 1000 / nsteps))
                                                     for v in drift],
               "sm_mhz": clocks.get("sm_mhz")}
        sec.update(counter_shares(st0, st1, int(fl.sum()) * args.steps))
        out[f"box{n}"] = sec
    out["note"] = ("FP32 populations stored as deviations from the rest equilibrium at "
                   "(rho, T) = (1, 0.5); the FP64 path it is compared with is parity-checked "
                   "against the FP64 oracle; mass and momentum drift relative to the total mass")
    return out


def root_finder_section(args, local, s, newton_mlups: float):
    """The other solvers of the constraint equations and stopping tolerances on the same
    input (the FP64 256^3 box) after the same steps: MLUPS, Newton updates per cell and the
    largest relative difference in rho/u/T from the Newton run's fields at 1e-12 (they solve
    every cell below the same residual, so only round-off and the looser tolerances differ)."""
    import numpy as np
    import torch

    from paper_1910_13515_gb300 import lbm39 as C
    from paper_1910_13515_gb300.lattice import Lattice
    out = {"newton_tol_1e-12_mlups": round(newton_mlups, 3)}
    ref = None
    fl = s.mask == 0
    for name, over in (("newton", {}), ("chord", {"root_finder": 1}),
                       ("fp32dir", {"root_finder": 2}), ("fp32start", {"root_finder": 3}),
                       ("newton_tol_1e-10", {"newton_tol": 1e-10}),
                       ("newton_tol_1e-8", {"newton_tol": 1e-8})):
        L = Lattice.from_setup(s, precision=C.LBM39_FP64, device=f"cuda:{local}", **over)
        c0 = L.stats().conserved
        L.step(args.warmup)
        st0 = L.stats()
        _, ms, _ = timed_steps(L, args.steps, local)
        st1 = L.stats()
        state = L.read_numpy()
        L.close()
        del L
        torch.cuda.empty_cache()
        if ref is None:
            ref = state
            if name == "newton":
                continue
        d = [float(np.abs(a[..., fl] - b[..., fl]).max() / max(np.abs(b[..., fl]).max(), 1e-300))
             for a, b in zip(state[:3], ref[:3])]
        out[name] = {"mlups": round(s.ncells * args.steps / (ms * 1e-3) / 1e6, 3),
                     "newton_updates_per_cell": round((st1.newton_updates - st0.newton_updates)
                                                      / (int(fl.sum()) * args.steps), 4),
                     **({"start32_steps_per_cell":
                         round((st1.start32_updates - st0.start32_updates)
                               / (int(fl.sum()) * args.steps), 4)}
                        if name == "fp32start" else {}),
                     "max_rel_diff_vs_newton_rho_u_T": [float("%.2e" % v) for v in d],
                     "conservation_drift_rel": [float("%.2e" % v)
                                                for v in drift_rel(c0, st1.conserved)]}
        out[name]["speedup_vs_newton"] = round(out[name]["mlups"] / newton_mlups, 3)
    return out


def prandtl_section(args, local, s, pr1_mlups: float):
    """The Prandtl-number adjustment (quasi-equilibrium collision, heat flux relaxed with
    tau2 = 1/2 + (tau_eff - 1/2)/Pr) on the same input (the FP64 256^3 box) after the same
    steps, at Pr = 0.71 (air) in both precisions: MLUPS, its ratio to the Pr = 1 step of the
    same precision (FP64: the line's value) and the conservation drift."""
    import torch

    from paper_1910_13515_gb300 import lbm39 as C
    from paper_1910_13515_gb300.lattice import Lattice
    out = {"prandtl": 0.71}
    fl = int((s.mask == 0).sum())
    base = {"fp64": pr1_mlups}
    for name, prec, pr in (("fp64", C.LBM39_FP64, 0.71), ("mixed_pr1", C.LBM39_MIXED, 1.0),
                           ("mixed", C.LBM39_MIXED, 0.71)):
        over = {"prandtl": pr} if pr != 1.0 else {}
        L = Lattice.from_setup(s, precision=prec, device=f"cuda:{local}", **over)
        c0 = L.stats().conserved
        L.step(args.warmup)
        st0 = L.stats()
        _, ms, _ = timed_steps(L, args.steps, local)
        st1 = L.stats()
        L.close()
        del L
        torch.cuda.empty_cache()
        mlups = round(s.ncells * args.steps / (ms * 1e-3) / 1e6, 3)
        if pr == 1.0:
            base["mixed"] = mlups
            continue
        out[name] = {"mlups": mlups, "vs_prandtl_1_same_precision": round(mlups / base[name], 3),
                     "fluid_cells": fl,
                     "newton_updates_per_cell": round((st1.newton_updates - st0.newton_updates)
                                                      / (fl * args.steps), 4),
                     "conservation_drift_rel": [float("%.2e" % v)
                                                for v in drift_rel(c0, st1.conserved)]}
    return out


def airfoil_section(args, local, developed_at: int):
    """The 2048x1024 NACA0012 airfoil (Ma 1.5, Re 1e4, C = 400), FP64: the rate over the early
    window of the impulsive start (steps W..W+K) and over K steps of the developed flow from
    step `developed_at` on (bow and trailing shocks formed), and the precision form over the
    early window."""
    from paper_1910_13515_gb300 import lbm39 as C
    from paper_1910_13515_gb300.lattice import Lattice
    s = make_setup("naca")
    L = Lattice.from_setup(s, precision=C.LBM39_FP64, device=f"cuda:{local}")
    fluid = int((s.mask == 0).sum())
    out = {"workload": WORKLOADS["naca"], "cells": s.ncells, "fluid_cells": fluid}
    L.step(args.warmup)
    L.sync()
    for name, t_start in (("early", args.warmup), ("developed", developed_at)):
        while L.time < t_start:
            L.step(min(500, t_start - L.time))
            L.sync()
        st0 = L.stats()
        _, ms, clocks = timed_steps(L, args.steps, local)
        L.sync()
        st1 = L.stats()
        sec = {"steps": [t_start, t_start + args.steps],
               "mlups": round(s.ncells * args.steps / (ms * 1e-3) / 1e6, 3),
               "fluid_mlups": round(fluid * args.steps / (ms * 1e-3) / 1e6, 3),
               "ms_per_step": round(ms / args.steps, 4), "sm_mhz": clocks.get("sm_mhz")}
        sec.update(counter_shares(st0, st1, fluid * args.steps))
        out[name] = sec
    L.close()
    # the precision form over the same early window, stored as deviations from the far-field
    # equilibrium (the Lattice default for a lattice with freestream cells)
    Lm = Lattice.from_setup(s, precision=C.LBM39_MIXED, device=f"cuda:{local}")
    Lm.step(args.warmup)
    Lm.sync()
    st0 = Lm.stats()
    _, ms, clocks = timed_steps(Lm, args.steps, local)
    Lm.sync()
    st1 = Lm.stats()
    sec = {"steps": [args.warmup, args.warmup + args.steps],
           "reference_state": "far field (rho, u, T) = (%g, %.4f, %g)" % (
               s.rho_inf, s.u_inf[0], s.T_inf),
           "mlups": round(s.ncells * args.steps / (ms * 1e-3) / 1e6, 3),
           "ms_per_step": round(ms / args.steps, 4), "sm_mhz": clocks.get("sm_mhz")}
    sec["speedup_vs_fp64_early"] = round(sec["mlups"] / out["early"]["mlups"], 3)
    sec.update(counter_shares(st0, st1, fluid * args.steps))
    out["precision_form_early"] = sec
    Lm.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="box256", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    ap.add_argument("--serve-rate", type=float, default=0.8)
    ap.add_argument("--mach", type=float, default=0.8,
                    help="box workloads: rms Mach number of the initial velocity field")
    ap.add_argument("--poly-n", type=int, default=2048,
                    help="poly workload: lattice side n of the periodic n x n x 1 lattice")
    ap.add_argument("--compare-fp64", action="store_true",
                    help="precision form: also run the FP64 path and report L1 error, drift, speedup")
    ap.add_argument("--sections", default="precision,serving,airfoil,root_finders,prandtl",
                    help="FP64 256^3 box line: comma-separated extra sections to run in the same "
                         "line (precision, serving, airfoil, root_finders, prandtl), or 'none'")
    ap.add_argument("--serve-requests", type=int, default=16,
                    help="requests of the serving section of the 256^3 box line")
    ap.add_argument("--serve-section-rate", type=float, default=3.0,
                    help="arrival rate (Hz) of the serving section: saturating by default")
    ap.add_argument("--developed-at", type=int, default=3000,
                    help="airfoil section: first step of the developed-flow window")
    ap.add_argument("--root-finder", default="newton",
                    choices=["newton", "chord", "fp32dir", "fp32start"],
                    help="solver of the constraint equations (chord: the chord-Newton hybrid; "
                         "fp32dir: Newton with a single-precision direction; fp32start: that "
                         "after a single-precision start)")
    ap.add_argument("--start-at", type=int, default=0,
                    help="step the lattice to this time before the warm-up (developed flows)")
    ap.add_argument("--checkpoint-out", default=None,
                    help="after --start-at, save the lattice's checkpoint (lbm39_save) to this file")
    ap.add_argument("--checkpoint-in", default=None,
                    help="start from a checkpoint saved with --checkpoint-out for the same "
                         "workload and options (instead of --start-at)")
    ap.add_argument("--newton-tol", type=float, default=1e-12,
                    help="stopping tolerance of the constraint solve (max |G_k| / rho)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "serve":
        run_serve(args, rank, world, local)
        return
    if args.workload == "poly":
        run_poly(args, rank, world, local)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_1910_13515_gb300 import lbm39 as C
    from paper_1910_13515_gb300.lattice import Lattice

    prec = C.LBM39_FP64 if args.precision == "fp64" else C.LBM39_MIXED
    s = make_setup(args.workload, args.mach)
    solver = {"root_finder": {"newton": 0, "chord": 1, "fp32dir": 2,
                              "fp32start": 3}[args.root_finder],
              "newton_tol": args.newton_tol}
    L = Lattice.from_setup(s, precision=prec, device=f"cuda:{local}", **solver)
    stream = L.stream
    N = s.ncells
    st_init = L.stats()
    fluid = st_init.fluid_cells
    if args.checkpoint_in:
        L.restore(torch.load(args.checkpoint_in).to(f"cuda:{local}"))
    while L.time < args.start_at:
        L.step(min(500, args.start_at - L.time))
        L.sync()
    if args.checkpoint_out:
        torch.save(L.checkpoint().cpu(), args.checkpoint_out)

    L.step(args.warmup)
    L.sync()
    st0 = L.stats()
    per_step, _, clocks = timed_steps(L, args.steps, local, barrier)
    elapsed_s, units = reduce_over_ranks(sum(per_step) * 1e-3, float(N * args.steps), dist,
                                         f"cuda:{local}")
    elapsed_ms = elapsed_s * 1e3
    L.sync()
    st1 = L.stats()
    cell_steps = fluid * args.steps
    shares = counter_shares(st0, st1, cell_steps)
    k_upd = shares["newton_updates_per_cell"]
    value = units / elapsed_s / 1e6
    headline_state = L.read_numpy()

    # dominant kernel (the fused step): per-launch duration on its own stream
    step_ms = float(np.mean(per_step))
    scratch = torch.empty(1 << 21, dtype=torch.float64, device=f"cuda:{local}")
    rc, peak_tf = C.lbm39_selftest_dfma(scratch.data_ptr(), scratch.numel() * 8,
                                        stream.cuda_stream)
    C.check(rc, "lbm39_selftest_dfma")
    del scratch
    # lattices one cell thick in z with u_z = 0 take the nine-constraint (z-mirror) solve
    reduced = (args.precision == "fp64" and s.nz == 1 and not np.any(s.u[2])
               and s.u_inf[2] == 0.0)
    model = FP64_FLOPS_MODEL.get(("fp64_2d" if reduced else args.precision)
                                 + ("" if args.root_finder == "newton" else "_" + args.root_finder))
    flops_cell = (model[0] + model[1] * k_upd
                  + (model[2] * shares["start32_solve_share"] if len(model) > 2 else 0.0)
                  if model else None)
    achieved_tf = flops_cell * fluid / (step_ms * 1e-3) / 1e12 if model else None
    hbm_gbs = BYTES_PER_UPDATE[args.precision] * fluid / (step_ms * 1e-3) / 1e9
    traffic = None
    if (NCU_TRAFFIC["kernel_hash"] == kernel_source_hash() and args.mach == 0.8
            and args.root_finder == "newton" and args.newton_tol == 1e-12):
        traffic = NCU_TRAFFIC["gb_per_launch"].get(f"{args.workload}/{args.precision}")
    roofline = {"bound": "alu", "achieved": round(achieved_tf, 4) if model else None,
                "peak": round(peak_tf, 4), "unit": "TFLOP/s",
                "frac": round(achieved_tf / peak_tf, 4) if model else None,
                "traffic": round(traffic * 1e9) if traffic else None,
                "peak_source": "FP64 FMA throughput measured in this run by lbm39_selftest_dfma "
                               "(of measured)",
                "flops_per_cell_update": round(flops_cell) if model else None,
                "flops_model": (f"{model[0]:g} + {model[1]:g} x (Newton updates per cell)"
                                + (f" + {model[2]:g} x (share of solves with a single-"
                                   "precision start)" if len(model) > 2 else "")
                                + ", fitted to ncu FP64 instruction counts (2 per DFMA, 1 per "
                                "DADD/DMUL)") if model else "none fitted for this solver",
                "hbm": {"achieved_gbs": round(hbm_gbs, 1), "peak_gbs": HBM_PEAK_GBS,
                        "frac": round(hbm_gbs / HBM_PEAK_GBS, 4),
                        "bytes_per_update": BYTES_PER_UPDATE[args.precision],
                        "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}}

    # end to end through the C ABI with host buffers: upload the initial fields from pinned
    # memory, then every step a step and a read-back of rho/u/T/p into pinned memory
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64)).pin_memory()
        h_rho, h_u, h_T = pin(s.rho), pin(s.u), pin(s.T)
        h_out = torch.empty((6, N), dtype=torch.float64).pin_memory()
        ke = args.steps
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        C.check(C.lbm39_init_host(L.h, h_rho.data_ptr(), h_u.data_ptr(), h_T.data_ptr()))
        for _ in range(ke):
            C.check(C.lbm39_step(L.h, 1))
            C.check(C.lbm39_read_host(L.h, h_out[0].data_ptr(), h_out[1].data_ptr(),
                                      h_out[4].data_ptr(), h_out[5].data_ptr()))
        dt, units_e2e = reduce_over_ranks(time.perf_counter() - t0, float(N * ke), dist,
                                          f"cuda:{local}")
        e2e = {"value": round(units_e2e / dt / 1e6, 3), "unit": "MLUPS",
               "h2d_bytes_per_step": int(5 * 8 * N / ke), "d2h_bytes_per_step": 6 * 8 * N,
               "steps": ke, "includes": "lbm39_init_host once (cold-start Newton) + per step "
                                       "lbm39_step(1) and lbm39_read_host of rho,u,T,p"}
        del h_rho, h_u, h_T, h_out
    launches = args.steps * (2 if L.has_fills else 1)

    # precision form against the FP64 path on the same input and step count (single run)
    form = None
    if args.compare_fp64 and prec == C.LBM39_MIXED:
        st_end = L.stats()
        L.close()
        Lf = Lattice.from_setup(s, precision=C.LBM39_FP64, device=f"cuda:{local}")
        Lf.step(args.warmup)
        _, ms, _ = timed_steps(Lf, args.steps, local)
        fp64_state = Lf.read_numpy()
        fp64_mlups = N * args.steps / (ms * 1e-3) / 1e6
        Lf.close()
        nsteps = args.warmup + args.steps
        drift = drift_rel(st_init.conserved, st_end.conserved)
        form = {"compared_after_steps": nsteps,
                "l1_rel_vs_fp64_rho_u_T": [float("%.3e" % v)
                                           for v in l1_rel(headline_state, fp64_state, s.mask == 0)],
                "conservation_drift_rel_mass_mom_xyz_energy": [float("%.3e" % v) for v in drift],
                "conservation_drift_per_1000_steps": [float("%.3e" % (v * 1000 / nsteps))
                                                      for v in drift],
                "fp64_mlups_same_run": round(fp64_mlups, 3),
                "speedup_vs_fp64": round(value / fp64_mlups, 3),
                "note": "FP64 path parity-checked against the FP64 oracle; mass and momentum "
                        "drift relative to the total mass"}
    else:
        L.close()
    del L
    torch.cuda.empty_cache()

    # the other parts of the metric, in the same line as the FP64 256^3 box
    sections = set() if args.sections == "none" else set(args.sections.split(","))
    suite = (args.workload == "box256" and args.precision == "fp64" and world == 1
             and args.root_finder == "newton" and args.newton_tol == 1e-12
             and args.start_at == 0 and not args.checkpoint_in)
    serving = airfoil = solvers = prandtl = None
    if suite and "precision" in sections:
        form = precision_form_section(args, local, s, (headline_state, value))
    del headline_state
    if suite and "root_finders" in sections:
        solvers = root_finder_section(args, local, s, value)
    if suite and "prandtl" in sections:
        prandtl = prandtl_section(args, local, s, value)
    if suite and "airfoil" in sections:
        airfoil = airfoil_section(args, local, args.developed_at)
    if suite and "serving" in sections:
        serving = serving_section(args, local, args.serve_requests, args.serve_section_rate)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        c, desc = crop_setup(s, args.workload)
        v, done, threads, dt = oracle_mlups(c, 10 ** 6, budget_s=args.cpu_budget_s)
        cpu = {"value": round(v, 4), "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": f"{desc}: {done} oracle steps in {dt:.1f} s (after its cold-start init)"}

    if rank == 0:
        config = {"workload": workload_text(args), "precision": args.precision,
                  "root_finder": args.root_finder, "newton_tol": args.newton_tol,
                  "timed_from_step": st0.time,
                  "cells": N, "fluid_cells": int(fluid),
                  "fluid_mlups": round(fluid * args.steps * world / (elapsed_ms * 1e-3) / 1e6, 3),
                  "l2": "inputs larger than L2 (%.2f GB of populations)" % (
                      BYTES_PER_UPDATE[args.precision] / 2 * N / 1e9),
                  "parallelism": "replicas" if world > 1 else "1 GPU"}
        config.update(shares)
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(elapsed_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32-storage/f64-solve",
            "data": "synthetic",
            "config": config,
            "clocks": clocks, "roofline": roofline, "e2e": e2e,
            "gpu_launches": launches,
            "cpu_baseline": cpu,
            "precision_form": form,
            "serving": serving,
            "airfoil": airfoil,
            "root_finders": solvers,
            "prandtl": prandtl,
            "kernel_hash": kernel_source_hash(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
