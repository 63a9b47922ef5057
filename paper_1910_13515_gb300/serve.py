"""Serving form: continuous batching of many lattice simulations on one GPU.

Requests (a Setup and a number of steps) arrive on a clock.  The scheduler
admits waiting requests whenever a slot and enough of the device-memory budget
are free, keeps admitted lattices resident, and advances all of them together
through lbm39_batch_run (one packed launch per time step, runs of graph_steps
steps replayed from a captured CUDA graph).  While a run is on the GPU the host
does not wait for it: it polls the run's completion event and meanwhile admits
the requests that arrive, creating and initialising their lattices on a second
stream, so that their set-up overlaps the running steps; they join the next
run.  A lattice that reaches its step count is read out and freed, which frees
memory for the next requests, so work that arrives while others run overlaps
with them on the device.  A request withdrawn by its client (Request.cancel_s)
is dropped if it is still waiting, or released at the next run boundary
(between steps) if it is resident; its memory goes to the next requests and the
report lists it with the steps it completed.  A request whose flow leaves the
13-moment cone is served like the others (its cells take the five-invariant
fallback); the report lists its fallback cell-steps (Report.failed).

Scheduler holds the policy and is independent of the GPU (a test drives it with a
fake backend); GpuBackend does the device work through the C ABI.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from .inputs import Request


@dataclass
class Job:
    req: Request
    bytes: int
    steps: int
    handle: object = None          # backend's lattice
    t_admit: float = 0.0
    t_done: float = 0.0
    result: tuple = None
    done_steps: int = 0


@dataclass
class Report:
    latencies_s: list
    wall_s: float
    cell_steps: int
    results: dict = field(default_factory=dict)
    max_resident: int = 0
    rounds: int = 0
    cancelled: dict = field(default_factory=dict)   # rid -> steps completed before withdrawal
    failed: dict = field(default_factory=dict)      # rid -> cell-steps that took the fallback

    @property
    def p50_ms(self) -> float:
        return float(np.percentile(self.latencies_s, 50) * 1e3)

    @property
    def p99_ms(self) -> float:
        return float(np.percentile(self.latencies_s, 99) * 1e3)

    @property
    def mlups(self) -> float:
        return self.cell_steps / self.wall_s / 1e6


class Scheduler:
    """Admission by memory budget and slots; run lengths bounded by the soonest finishing
    resident job and by `chunk_steps` (so new arrivals wait at most one chunk)."""

    def __init__(self, backend, budget_bytes: int, max_resident: int, chunk_steps: int = 64,
                 clock=time.perf_counter, sleep=time.sleep, poll_s: float = 2e-4):
        self.be = backend
        self.budget = budget_bytes
        self.max_resident = max_resident
        self.chunk = chunk_steps
        self.clock = clock
        self.sleep = sleep
        self.poll_s = poll_s

    def run(self, requests) -> Report:
        pending = deque(sorted(requests, key=lambda r: r.arrival_s))
        for r in pending:
            if self.be.bytes_for(r.setup) > self.budget:
                raise ValueError(f"request {r.rid} needs more than the whole memory budget")
        waiting: deque = deque()
        active: list = []      # resident and in the batch
        incoming: list = []    # admitted while a run was on the GPU: join the next run
        done: dict = {}
        cancelled: dict = {}
        used = 0
        t0 = self.clock()
        max_res = 0
        rounds = 0
        busy = getattr(self.be, "busy", None)   # asynchronous backends only
        wait = getattr(self.be, "wait", None)
        failed_of = getattr(self.be, "failed", None)
        failed: dict = {}

        def arrivals(now):
            while pending and pending[0].arrival_s <= now:
                r = pending.popleft()
                waiting.append(Job(r, self.be.bytes_for(r.setup), r.setup.steps))

        def admit_into(dest, now_fn) -> bool:
            nonlocal used
            admitted = False
            while waiting and len(active) + len(incoming) < self.max_resident and \
                    used + waiting[0].bytes <= self.budget:
                j = waiting.popleft()
                j.handle = self.be.admit(j.req.setup)
                j.t_admit = now_fn()
                used += j.bytes
                dest.append(j)
                admitted = True
            return admitted

        while pending or waiting or active or incoming:
            now = self.clock() - t0
            arrivals(now)
            if incoming:
                active.extend(incoming)
                incoming.clear()
                self.be.needs_set = True
            # withdrawals: waiting jobs are dropped, resident ones released between steps
            gone = [j for j in waiting if _withdrawn(j, now)]
            for j in gone:
                waiting.remove(j)
                cancelled[j.req.rid] = 0
            gone = [j for j in active if _withdrawn(j, now)]
            for j in gone:
                self.be.release(j.handle)
                used -= j.bytes
                cancelled[j.req.rid] = j.done_steps
                active.remove(j)
                self.be.needs_set = True
            admitted = admit_into(active, lambda: self.clock() - t0)
            max_res = max(max_res, len(active))
            if not active:
                if pending:  # idle until the next arrival
                    self.sleep(max(0.0, pending[0].arrival_s - (self.clock() - t0)))
                continue
            if admitted or self.be.needs_set:
                self.be.set_resident([j.handle for j in active], [j.steps for j in active])
            n = min(self.chunk, min(j.steps - j.done_steps for j in active))
            self.be.run(n)
            rounds += 1
            # while the run is on the GPU: admit what arrives (set up on the side)
            while busy is not None and busy():
                arrivals(self.clock() - t0)
                if not admit_into(incoming, lambda: self.clock() - t0):
                    self.sleep(self.poll_s)
                max_res = max(max_res, len(active) + len(incoming))
            if wait is not None:
                wait()
            for j in active:
                j.done_steps += n
            finished = [j for j in active if j.done_steps >= j.steps]
            if finished:
                for j in finished:
                    j.result = self.be.read(j.handle)
                    nf = failed_of(j.handle) if failed_of is not None else 0
                    if nf:
                        failed[j.req.rid] = nf
                    j.t_done = self.clock() - t0
                    self.be.release(j.handle)
                    used -= j.bytes
                    done[j.req.rid] = j
                active = [j for j in active if j.done_steps < j.steps]
                self.be.needs_set = True
        if done:
            wall = max(j.t_done for j in done.values()) - min(j.req.arrival_s for j in done.values())
        else:
            wall = 0.0
        lat = [j.t_done - j.req.arrival_s for j in done.values()]
        cells = sum(j.req.setup.ncells * j.steps for j in done.values())
        return Report(lat, wall, cells, {rid: j.result for rid, j in done.items()}, max_res,
                      rounds, cancelled, failed)


def _withdrawn(job: Job, now: float) -> bool:
    c = getattr(job.req, "cancel_s", None)
    return c is not None and c <= now


class GpuBackend:
    """Lattices on one GPU, advanced together by a batch of the C ABI.  The batch runs on its
    own stream; lattices are created, initialised and read out on a second stream, so that
    admissions overlap a running batch.  run() returns once the steps are enqueued; busy()
    polls their completion event and wait() blocks on it."""

    def __init__(self, precision=0, max_lattices: int = 64, max_cells: int = 1 << 25,
                 graph_steps: int = 8, device="cuda"):
        import torch

        from . import lbm39 as C
        self.torch, self.C = torch, C
        self.device = torch.device(device)
        # graph capture needs a created stream (not the legacy default stream)
        self.stream = torch.cuda.Stream(self.device)
        self.side = torch.cuda.Stream(self.device)   # admissions and read-outs
        self.precision = precision
        rc, nbytes = C.lbm39_batch_query_bytes(max_lattices, max_cells)
        C.check(rc, "lbm39_batch_query_bytes")
        self.buf = torch.empty((nbytes + 7) // 8, dtype=torch.float64, device=self.device)
        rc, self.b = C.lbm39_batch_create(max_lattices, max_cells, precision, graph_steps,
                                          self.buf.data_ptr(), self.stream.cuda_stream)
        C.check(rc, "lbm39_batch_create")
        self.needs_set = True
        self.done_ev = None

    def bytes_for(self, setup) -> int:
        from .lattice import params_from_setup
        rc, pop, aux = self.C.lbm39_query_bytes(params_from_setup(setup, self.precision))
        self.C.check(rc, "lbm39_query_bytes")
        return pop + aux + setup.ncells

    def admit(self, setup):
        """Creates and initialises the request's lattice on the side stream (lbm39_init waits
        for its own work only), while a batch run may still be on the GPU."""
        from .lattice import Lattice
        return Lattice.from_setup(setup, precision=self.precision, device=self.device,
                                  stream=self.side)

    def set_resident(self, lattices, steps):
        # every lattice starts at time 0, so its end time is its step count
        self.C.check(self.C.lbm39_batch_set(self.b, [L.h for L in lattices], list(steps)),
                     "lbm39_batch_set")
        self.needs_set = False

    def run(self, n: int):
        self.C.check(self.C.lbm39_batch_run(self.b, n), "lbm39_batch_run")
        self.done_ev = self.torch.cuda.Event()
        self.done_ev.record(self.stream)

    def busy(self) -> bool:
        return self.done_ev is not None and not self.done_ev.query()

    def wait(self):
        if self.done_ev is not None:
            self.done_ev.synchronize()

    def read(self, L):
        """The finished lattice's rho, u, T, p.  Cells whose constraint solve failed took the
        five-invariant fallback (a valid, conservative state): failed(L) reports how many
        cell-steps did, so one request leaving the moment cone does not stop the others."""
        self.wait()
        L.served_failed = L.sync()
        return L.read_numpy()

    def failed(self, L) -> int:
        """Cell-steps of the lattice that took the fallback equilibrium (after read)."""
        return int(getattr(L, "served_failed", 0))

    def release(self, L):
        self.wait()
        L.close()
        L.pop = L.aux = L.mask = None

    def close(self):
        if getattr(self, "b", None):
            self.wait()
            self.C.lbm39_batch_destroy(self.b)
            self.b = None
