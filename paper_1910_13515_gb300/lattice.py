"""Lattice: one D3Q39 DDF lattice on one GPU, over torch-allocated device buffers.

PyTorch provides the device memory and the stream; every computation is a
kernel of liblbm39 called through the C ABI (``lbm39`` module).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import lbm39 as C
from .inputs import M_FREE, Setup


def velocities():
    """(vel (39,3) int32, w (39,) float64) in the library's population order."""
    vel = np.zeros((C.Q, 3), np.int32)
    w = np.zeros(C.Q)
    C.check(C.lbm39_velocities(vel.ctypes.data, w.ctypes.data), "lbm39_velocities")
    return vel, w


def params_from_setup(s: Setup, precision: int = C.LBM39_FP64, **over) -> C.lbm39_params:
    """Run parameters of a setup.  The precision form of a lattice with freestream cells
    stores its populations as deviations from the far-field equilibrium (ref_rho, ref_u,
    ref_T = rho_inf, u_inf, T_inf), so that the flow that moves with the far field is stored
    finely; other lattices keep the library's rest reference (1, 0, 0.5).  Keyword
    arguments override any field."""
    p = C.lbm39_default_params(s.nx, s.ny, s.nz)
    for a in range(3):
        p.periodic[a] = int(s.periodic[a])
        p.u_inf[a] = float(s.u_inf[a])
    p.gamma = s.gamma
    p.tau = s.tau
    p.kn_sensor = int(s.kn_sensor)
    p.rho_inf = s.rho_inf
    p.T_inf = s.T_inf
    p.precision = precision
    if precision == C.LBM39_MIXED and s.mask is not None and \
            bool((np.asarray(s.mask) == M_FREE).any()):
        p.ref_rho, p.ref_T = s.rho_inf, s.T_inf
        for a in range(3):
            p.ref_u[a] = float(s.u_inf[a])
    for k, v in over.items():
        setattr(p, k, v)
    return p


class Guarded:
    """A float64 buffer of n elements between two 64 KiB canary zones (a fixed bit pattern),
    for debug runs: a kernel write before the start or past the end changes a canary.  The
    buffer keeps the 256-byte alignment of the allocation."""

    PAD = 8192                      # float64 elements per zone (64 KiB)
    PATTERN = 0x7FF4C0DEC0DE5A5A    # a signalling-NaN bit pattern no kernel writes

    def __init__(self, n: int, device):
        self.full = torch.empty(n + 2 * self.PAD, dtype=torch.float64, device=device)
        self.full[:self.PAD].view(torch.int64).fill_(self.PATTERN)
        self.full[self.PAD + n:].view(torch.int64).fill_(self.PATTERN)
        self.buf = self.full[self.PAD:self.PAD + n]

    def intact(self) -> bool:
        head = self.full[:self.PAD].view(torch.int64)
        tail = self.full[self.PAD + self.buf.numel():].view(torch.int64)
        return bool((head == self.PATTERN).all()) and bool((tail == self.PATTERN).all())


def _buffers(pop_b: int, aux_b: int, device, debug: bool):
    """(pop, aux) float64 device buffers of at least the given byte sizes, canary-guarded in
    debug mode (then also the Guarded objects, else None)."""
    n_pop, n_aux = (pop_b + 7) // 8, (aux_b + 7) // 8
    if not debug:
        return (torch.empty(n_pop, dtype=torch.float64, device=device),
                torch.empty(n_aux, dtype=torch.float64, device=device), None)
    g = (Guarded(n_pop, device), Guarded(n_aux, device))
    return g[0].buf, g[1].buf, g


def _check_guards(guards, where: str):
    if guards is None:
        return
    if guards[0].full.is_cuda:
        torch.cuda.synchronize(guards[0].full.device)
    for name, g in zip(("population", "auxiliary"), guards):
        if not g.intact():
            raise RuntimeError(f"{where}: a kernel wrote outside the {name} buffer")


class Lattice:
    """Owns the device buffers of one lattice and its library handle.  debug=True puts
    canary zones around the population and auxiliary buffers and checks them after every
    init and step call (with a device synchronisation)."""

    def __init__(self, params: C.lbm39_params, mask: np.ndarray | None = None,
                 device: str | torch.device = "cuda", stream: torch.cuda.Stream | None = None,
                 debug: bool = False):
        self.params = params
        self.device = torch.device(device)
        self.N = params.nx * params.ny * params.nz
        rc, pop_b, aux_b = C.lbm39_query_bytes(params)
        C.check(rc, "lbm39_query_bytes")
        # 256-byte aligned by the caching allocator; float64 storage keeps 8-byte units
        self.pop, self.aux, self._guards = _buffers(pop_b, aux_b, self.device, debug)
        self.mask = None
        # freestream, outflow or solid cells: the library runs a fill kernel after each pass
        self.has_fills = mask is not None and bool(
            np.isin(np.asarray(mask), (1, 2, 3)).any())
        if mask is not None:
            self.mask = torch.as_tensor(np.ascontiguousarray(mask, np.uint8).reshape(-1),
                                        device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        vel, w = velocities()
        self._vel, self._w = vel, w
        rc, h = C.lbm39_create(params, vel.ctypes.data, w.ctypes.data, self.pop.data_ptr(),
                               self.aux.data_ptr(),
                               self.mask.data_ptr() if self.mask is not None else None,
                               self.stream.cuda_stream)
        C.check(rc, "lbm39_create")
        self.h = h

    @classmethod
    def from_setup(cls, s: Setup, precision: int = C.LBM39_FP64, device="cuda", stream=None,
                   debug: bool = False, **over) -> "Lattice":
        L = cls(params_from_setup(s, precision, **over), s.mask, device, stream, debug)
        L.init(s.rho, s.u, s.T)
        return L

    def close(self):
        if getattr(self, "h", None):
            C.lbm39_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state -----------------------------------------------------------------------------
    def _dev(self, a, n):
        t = torch.as_tensor(np.ascontiguousarray(a, np.float64).reshape(-1), device=self.device) \
            if not isinstance(a, torch.Tensor) else a.to(self.device, torch.float64).contiguous()
        assert t.numel() == n
        return t

    def init(self, rho, u, T):
        r, uu, t = self._dev(rho, self.N), self._dev(u, 3 * self.N), self._dev(T, self.N)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        C.check(C.lbm39_init(self.h, r.data_ptr(), uu.data_ptr(), t.data_ptr()), "lbm39_init")
        self._keep = (r, uu, t)  # alive until the kernels have read them
        self.sync()
        _check_guards(self._guards, "lbm39_init")

    def init_host(self, rho, u, T):
        """Initial condition from host arrays (copied through the library's staging)."""
        r = np.ascontiguousarray(rho, np.float64)
        uu = np.ascontiguousarray(u, np.float64)
        t = np.ascontiguousarray(T, np.float64)
        C.check(C.lbm39_init_host(self.h, r.ctypes.data, uu.ctypes.data, t.ctypes.data),
                "lbm39_init_host")

    def step(self, n: int = 1):
        C.check(C.lbm39_step(self.h, int(n)), "lbm39_step")
        _check_guards(self._guards, "lbm39_step")

    def sync(self, timeout_us: int = -1) -> int:
        rc, failed = C.lbm39_sync(self.h, timeout_us)
        if rc not in (C.LBM39_OK, C.LBM39_ERR_NEWTON):
            C.check(rc, "lbm39_sync")
        return failed

    def read(self):
        """(rho, u (3,N), T, p) as float64 device tensors."""
        out = torch.empty(6, self.N, dtype=torch.float64, device=self.device)
        C.check(C.lbm39_read(self.h, out[0].data_ptr(), out[1].data_ptr(), out[4].data_ptr(),
                             out[5].data_ptr()), "lbm39_read")
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return out[0], out[1:4], out[4], out[5]

    def read_numpy(self):
        r, u, T, p = self.read()
        self.stream.synchronize()
        return r.cpu().numpy(), u.cpu().numpy(), T.cpu().numpy(), p.cpu().numpy()

    def read_host(self, out: np.ndarray | None = None):
        """Host read-out through the library's staging: (rho, u, T, p) numpy arrays."""
        if out is None:
            out = np.empty((6, self.N))
        C.check(C.lbm39_read_host(self.h, out[0].ctypes.data, out[1].ctypes.data,
                                  out[4].ctypes.data, out[5].ctypes.data), "lbm39_read_host")
        return out[0], out[1:4], out[4], out[5]

    def diag_fields(self):
        """(eps float64, n_upd int32) device tensors of the current state: the Knudsen sensor
        and the Newton updates the next step takes (-1: the solve fails); state unchanged."""
        eps = torch.empty(self.N, dtype=torch.float64, device=self.device)
        nupd = torch.empty(self.N, dtype=torch.int32, device=self.device)
        C.check(C.lbm39_diag_fields(self.h, eps.data_ptr(), nupd.data_ptr()),
                "lbm39_diag_fields")
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return eps, nupd

    def stats(self) -> C.lbm39_stats_t:
        rc, s = C.lbm39_stats(self.h)
        C.check(rc, "lbm39_stats")
        return s

    def checkpoint(self) -> torch.Tensor:
        n = C.lbm39_checkpoint_bytes(self.h)
        buf = torch.empty(n, dtype=torch.uint8, device=self.device)
        C.check(C.lbm39_save(self.h, buf.data_ptr()), "lbm39_save")
        return buf

    def restore(self, buf: torch.Tensor):
        C.check(C.lbm39_load(self.h, buf.data_ptr()), "lbm39_load")

    @property
    def time(self) -> int:
        return int(self.stats().time)


class PolyLattice:
    """One periodic lattice of the polynomial-equilibrium comparison model (lbm39_poly.h):
    D3Q39 DDF-BGK with the fourth-order Hermite equilibrium, FP64, over torch buffers."""

    def __init__(self, nx: int, ny: int, nz: int, gamma: float = 1.4, tau: float = 0.6,
                 device: str | torch.device = "cuda", stream: torch.cuda.Stream | None = None,
                 debug: bool = False):
        p = C.lbm39_default_params(nx, ny, nz)
        p.kn_sensor = 0
        p.gamma = gamma
        p.tau = tau
        self.params = p
        self._debug = debug
        self.device = torch.device(device)
        self.N = nx * ny * nz
        rc, pop_b, aux_b = C.lbm39_poly_query_bytes(p)
        C.check(rc, "lbm39_poly_query_bytes")
        self.pop, self.aux, self._guards = _buffers(pop_b, aux_b, self.device, self._debug)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        rc, h = C.lbm39_poly_create(p, self.pop.data_ptr(), self.aux.data_ptr(),
                                    self.stream.cuda_stream)
        C.check(rc, "lbm39_poly_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            C.lbm39_poly_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, a, n):
        t = torch.as_tensor(np.ascontiguousarray(a, np.float64).reshape(-1), device=self.device) \
            if not isinstance(a, torch.Tensor) else a.to(self.device, torch.float64).contiguous()
        assert t.numel() == n
        return t

    def init(self, rho, u, T):
        r, uu, t = self._dev(rho, self.N), self._dev(u, 3 * self.N), self._dev(T, self.N)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        C.check(C.lbm39_poly_init(self.h, r.data_ptr(), uu.data_ptr(), t.data_ptr()),
                "lbm39_poly_init")
        self.stream.synchronize()  # the kernel has read r, uu, t
        _check_guards(self._guards, "lbm39_poly_init")

    def step(self, n: int = 1):
        C.check(C.lbm39_poly_step(self.h, int(n)), "lbm39_poly_step")
        _check_guards(self._guards, "lbm39_poly_step")

    def read(self):
        """(rho, u (3,N), T, p) as float64 device tensors."""
        out = torch.empty(6, self.N, dtype=torch.float64, device=self.device)
        C.check(C.lbm39_poly_read(self.h, out[0].data_ptr(), out[1].data_ptr(),
                                  out[4].data_ptr(), out[5].data_ptr()), "lbm39_poly_read")
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return out[0], out[1:4], out[4], out[5]

    def read_numpy(self):
        r, u, T, p = self.read()
        self.stream.synchronize()
        return r.cpu().numpy(), u.cpu().numpy(), T.cpu().numpy(), p.cpu().numpy()

    def conserved(self) -> np.ndarray:
        """[mass, momentum x/y/z, total energy] (waits for the stream)."""
        s = np.zeros(5)
        C.check(C.lbm39_poly_conserved(self.h, s.ctypes.data), "lbm39_poly_conserved")
        return s

    @property
    def time(self) -> int:
        return int(C.lbm39_poly_time(self.h))
