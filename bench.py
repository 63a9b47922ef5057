#!/usr/bin/env python
"""Benchmark of the D3Q39 13-moment DDF lattice Boltzmann step (MLUPS) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload naca|box256|box384|sod] [--precision fp64|mixed]

A step is one full time step (collide + stream with the mask rules) over the whole
lattice.  Inputs are synthetic and seeded (paper_1910_13515_gb300.inputs).  For N > 1
(torchrun, one process per GPU) every rank runs its own replica of the workload
(weak scaling; the step has no exchange between replicas).  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
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
    "sod": "Sod tube 400x1x1, outflow ends, tau=0.5 with alpha(eps)",
}

# FP64 arithmetic of one fluid-cell update as executed by the step kernel, from ncu
# instruction counts (2 flops per DFMA, 1 per DADD/DMUL): A + B * (Newton updates per cell)
# + C * (extra equilibrium evaluations of the line search, per cell).  See profiles/.
FP64_FLOPS_MODEL = {"fp64": (0.0, 0.0, 0.0), "mixed": (0.0, 0.0, 0.0)}
FP64_PEAK_TFLOPS = 1.008   # measured DFMA throughput (own microbenchmark), profiles/
BYTES_PER_UPDATE = {"fp64": 78 * 8 * 2 + 13 * 8 * 2, "mixed": 78 * 4 * 2 + 13 * 8 * 2}


def make_setup(name: str):
    from paper_1910_13515_gb300 import inputs
    if name == "naca":
        return inputs.naca()
    if name == "box256":
        return inputs.box(n=256, seed=0)
    if name == "box384":
        return inputs.box(n=384, seed=0)
    if name == "box128":
        return inputs.box(n=128, seed=0)
    if name == "sod":
        return inputs.sod(400)
    raise ValueError(name)


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


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle as it stands, on the host cores, each step a
    bounded sample (a window) of the same workload."""
    if rank != 0:
        return
    s = make_setup(args.workload)
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
            "config": {"workload": WORKLOADS[args.workload] + f" [oracle on a {desc}]",
                       "cells": c.ncells},
            "cpu_baseline": {"value": round(v, 4), "unit": "MLUPS", "cores": threads,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": round(v, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="naca", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
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
    s = make_setup(args.workload)
    L = Lattice.from_setup(s, precision=prec, device=f"cuda:{local}")
    stream = L.stream
    N = s.ncells
    fluid = L.stats().fluid_cells

    L.step(args.warmup)
    if L.sync() != 0:
        raise RuntimeError("Newton failures during warm-up")
    st0 = L.stats()

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
    elapsed_ms = evs[0].elapsed_time(evs[-1])
    t = torch.tensor([elapsed_ms], device=f"cuda:{local}")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    elapsed_ms = float(t.item())
    if L.sync() != 0:
        raise RuntimeError("Newton failures in the timed region")
    st1 = L.stats()
    cell_steps = fluid * args.steps
    k_upd = (st1.newton_updates - st0.newton_updates) / cell_steps
    value = N * args.steps * world / (elapsed_ms * 1e-3) / 1e6

    # dominant kernel (the fused step): per-launch duration on its own stream
    step_ms = float(np.mean(per_step))
    A, B, Cc = FP64_FLOPS_MODEL[args.precision]
    flops_cell = A + B * k_upd
    achieved_tf = flops_cell * fluid / (step_ms * 1e-3) / 1e12 if flops_cell > 0 else None
    roofline = {"bound": "alu", "achieved": round(achieved_tf, 4) if achieved_tf else None,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": round(achieved_tf / FP64_PEAK_TFLOPS, 4) if achieved_tf else None,
                "traffic": None,
                "peak_source": "measured DFMA throughput (of measured)",
                "hbm_gbs": round(BYTES_PER_UPDATE[args.precision] * fluid / (step_ms * 1e-3) / 1e9, 1)}

    # end to end through the C ABI with host buffers: upload the initial fields from pinned
    # memory, then every step a step and a read-back of rho/u/T/p into pinned memory
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64)).pin_memory()
        h_rho, h_u, h_T = pin(s.rho), pin(s.u), pin(s.T)
        h_out = torch.empty((6, N), dtype=torch.float64).pin_memory()
        ke = max(4, args.steps // 4)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        C.check(C.lbm39_init_host(L.h, h_rho.data_ptr(), h_u.data_ptr(), h_T.data_ptr()))
        for _ in range(ke):
            C.check(C.lbm39_step(L.h, 1))
            C.check(C.lbm39_read_host(L.h, h_out[0].data_ptr(), h_out[1].data_ptr(),
                                      h_out[4].data_ptr(), h_out[5].data_ptr()))
        dt = time.perf_counter() - t0
        tt = torch.tensor([dt], device=f"cuda:{local}")
        if world > 1:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dt = float(tt.item())
        e2e = {"value": round(N * ke * world / dt / 1e6, 3), "unit": "MLUPS",
               "h2d_bytes_per_step": int(5 * 8 * N / ke), "d2h_bytes_per_step": 6 * 8 * N,
               "steps": ke, "includes": "lbm39_init_host once (cold-start Newton) + per step "
                                       "lbm39_step(1) and lbm39_read_host of rho,u,T,p"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        c, desc = crop_setup(s, args.workload)
        v, done, threads, dt = oracle_mlups(c, 10 ** 6, budget_s=args.cpu_budget_s)
        cpu = {"value": round(v, 4), "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": f"{desc}: {done} oracle steps in {dt:.1f} s (after its cold-start init)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(elapsed_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32-storage/f64-solve",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "precision": args.precision,
                       "cells": N, "fluid_cells": int(fluid),
                       "fluid_mlups": round(fluid * args.steps * world / (elapsed_ms * 1e-3) / 1e6, 3),
                       "newton_updates_per_cell": round(k_upd, 4),
                       "l2": "inputs larger than L2 (%.2f GB of populations)" % (
                           BYTES_PER_UPDATE[args.precision] / 2 * N / 1e9),
                       "parallelism": "replicas" if world > 1 else "1 GPU"},
            "clocks": clocks, "roofline": roofline, "e2e": e2e,
            "gpu_launches": args.steps * (2 if L.has_ghosts else 1),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    L.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
