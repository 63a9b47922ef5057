"""ctypes wrapper of the plain FP64 CPU oracle (``oracle39.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library never
imports this module and this module never imports the CUDA library.

Paper: Latt, Coreixas, Beny, Parmigiani, arXiv:1910.13515 -- Sec. 2 (13-moment
exponential equilibrium, Eq. discrete-equilibrium, Eq. 13constraints), Sec. 3
(D3Q39, Newton-Raphson, BGK collide-and-stream, Eq. DeltaAvg and Eq. alpha),
Sec. 5 (the equilibrium step table).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle39.c")
_LIB = os.path.join(_HERE, "liboracle39.so")

Q = 39
NM = 13

M_FLUID, M_SOLID, M_FREE, M_OUT = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile oracle39.c into liboracle39.so with gcc (OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("periodic", ctypes.c_int32 * 3),
        ("gamma", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("kn_sensor", ctypes.c_int32),
        ("newton_tol", ctypes.c_double),
        ("newton_maxit", ctypes.c_int32),
        ("newton_min_upd", ctypes.c_int32),
        ("rho_inf", ctypes.c_double),
        ("u_inf", ctypes.c_double * 3),
        ("T_inf", ctypes.c_double),
        ("prandtl", ctypes.c_double),
        ("root_finder", ctypes.c_int32),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("fluid_cells", ctypes.c_int64),
        ("failed_cells", ctypes.c_int64),
        ("newton_updates", ctypes.c_int64),
        ("hist", ctypes.c_int64 * 32),
        ("eps_hist", ctypes.c_int64 * 4),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i32, i64, vp = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        P = ctypes.POINTER(Params)
        _lib.o39_lattice.argtypes = [vp, vp, vp]
        _lib.o39_lattice.restype = ctypes.c_int
        _lib.o39_basis.argtypes = [vp, vp]
        _lib.o39_targets.argtypes = [vp, d, vp]
        _lib.o39_feq_norm.argtypes = [vp, vp]
        _lib.o39_residual.argtypes = [vp, vp, vp]
        _lib.o39_jacobian.argtypes = [vp, vp]
        _lib.o39_invert.argtypes = [vp, vp]
        _lib.o39_invert.restype = ctypes.c_int
        _lib.o39_gaussian_guess.argtypes = [vp, d, vp]
        _lib.o39_newton.argtypes = [vp, vp, d, ctypes.c_int, ctypes.c_int, vp, vp]
        _lib.o39_newton.restype = ctypes.c_int
        _lib.o39_newton_hybrid.argtypes = [vp, vp, d, ctypes.c_int, ctypes.c_int, vp, vp, vp]
        _lib.o39_newton_hybrid.restype = ctypes.c_int
        _lib.o39_newton_fp32dir.argtypes = [vp, vp, d, ctypes.c_int, ctypes.c_int, vp, vp]
        _lib.o39_newton_fp32dir.restype = ctypes.c_int
        _lib.o39_newton_fp32start.argtypes = [vp, vp, d, ctypes.c_int, ctypes.c_int, vp, vp, vp]
        _lib.o39_newton_fp32start.restype = ctypes.c_int
        _lib.o39_alpha.argtypes = [d, d]
        _lib.o39_alpha.restype = d
        _lib.o39_cell_macros.argtypes = [P, vp, vp, vp, vp, vp]
        _lib.o39_newton5.argtypes = [vp, vp, d, ctypes.c_int, vp, vp]
        _lib.o39_newton5.restype = ctypes.c_int
        _lib.o39_targets5.argtypes = [vp, d, vp]
        _lib.o39_targets5.restype = None
        _lib.o39_gaussian_guess5.argtypes = [vp, d, vp]
        _lib.o39_gaussian_guess5.restype = None
        _lib.o39_collide_cell.argtypes = [P, vp, vp, vp, vp, i64, vp, vp, vp]
        _lib.o39_collide_cell.restype = ctypes.c_int
        _lib.o39_equilibrium.argtypes = [P, d, vp, d, vp, vp, vp, ctypes.c_int, vp]
        _lib.o39_equilibrium.restype = ctypes.c_int
        _lib.o39_init.argtypes = [P, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_int]
        _lib.o39_init.restype = i64
        _lib.o39_stream.argtypes = [P, vp, vp, vp, vp, vp, vp, vp]
        _lib.o39_step.argtypes = [P, vp, vp, vp, vp, vp, i64, ctypes.c_int, ctypes.POINTER(Stats)]
        _lib.o39_step.restype = i64
        _lib.o39_macros.argtypes = [P, vp, vp, vp, vp, vp, vp, vp]
        _lib.o39_conserved.argtypes = [P, vp, vp, vp, vp]
        del i32
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# Per-cell functions.

def lattice():
    """D3Q39 velocities (39,3) int32, Shan weights (39,), opposite index (39,)."""
    vel = np.zeros((Q, 3), np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, np.int32)
    n = lib().o39_lattice(_p(vel), _p(w), _p(opp))
    assert n == Q
    return vel, w, opp


def basis(xi) -> np.ndarray:
    xi = np.ascontiguousarray(xi, dtype=np.int32)
    out = np.zeros(NM)
    lib().o39_basis(_p(xi), _p(out))
    return out


def targets(u, T) -> np.ndarray:
    out = np.zeros(NM)
    lib().o39_targets(_p(_f64(u)), float(T), _p(out))
    return out


def feq_norm(lam) -> np.ndarray:
    out = np.zeros(Q)
    lib().o39_feq_norm(_p(_f64(lam)), _p(out))
    return out


def residual(lam, m) -> np.ndarray:
    out = np.zeros(NM)
    lib().o39_residual(_p(_f64(lam)), _p(_f64(m)), _p(out))
    return out


def jacobian(lam) -> np.ndarray:
    out = np.zeros((NM, NM))
    lib().o39_jacobian(_p(_f64(lam)), _p(out))
    return out


def invert(J) -> np.ndarray:
    out = np.zeros((NM, NM))
    rc = lib().o39_invert(_p(_f64(J)), _p(out))
    if rc != 0:
        raise np.linalg.LinAlgError("singular")
    return out


def gaussian_guess(u, T) -> np.ndarray:
    out = np.zeros(NM)
    lib().o39_gaussian_guess(_p(_f64(u)), float(T), _p(out))
    return out


def newton(m, lam0, tol=1e-12, maxit=30, min_upd=0):
    """Returns (lam, F, n_updates, status)."""
    lam = _f64(lam0).copy()
    F = np.zeros(Q)
    nu = ctypes.c_int(0)
    st = lib().o39_newton(_p(_f64(m)), _p(lam), float(tol), int(maxit), int(min_upd),
                          ctypes.byref(nu), _p(F))
    return lam, F, nu.value, st


def newton_hybrid(m, lam0, tol=1e-12, maxit=30, min_upd=0):
    """The chord-Newton hybrid: (lam, F, n_updates, n_jacobians, status)."""
    lam = _f64(lam0).copy()
    F = np.zeros(Q)
    nu = ctypes.c_int(0)
    nj = ctypes.c_int(0)
    st = lib().o39_newton_hybrid(_p(_f64(m)), _p(lam), float(tol), int(maxit), int(min_upd),
                                 ctypes.byref(nu), ctypes.byref(nj), _p(F))
    return lam, F, nu.value, nj.value, st


def newton_fp32dir(m, lam0, tol=1e-12, maxit=30, min_upd=0):
    """Newton with a single-precision direction: (lam, F, n_updates, status)."""
    lam = _f64(lam0).copy()
    F = np.zeros(Q)
    nu = ctypes.c_int(0)
    st = lib().o39_newton_fp32dir(_p(_f64(m)), _p(lam), float(tol), int(maxit), int(min_upd),
                                  ctypes.byref(nu), _p(F))
    return lam, F, nu.value, st


def targets5(u, T) -> np.ndarray:
    out = np.zeros(5)
    lib().o39_targets5(_p(_f64(u)), float(T), _p(out))
    return out


def newton5(u, T, tol=1e-12, maxit=50):
    """Fallback equilibrium of (u, T) (five collision invariants) from the Gaussian start:
    (mu, F, n_updates, status)."""
    m = targets5(u, T)
    mu = np.zeros(5)
    lib().o39_gaussian_guess5(_p(_f64(u)), float(T), _p(mu))
    F = np.zeros(Q)
    nu = ctypes.c_int(0)
    st = lib().o39_newton5(_p(m), _p(mu), float(tol), int(maxit), ctypes.byref(nu), _p(F))
    return mu, F, nu.value, st


def alpha(eps, tau) -> float:
    return lib().o39_alpha(float(eps), float(tau))


@dataclass
class Config:
    """Lattice and run parameters of the oracle (its own mirror of the method's inputs)."""
    nx: int
    ny: int = 1
    nz: int = 1
    periodic: tuple = (1, 1, 1)
    gamma: float = 1.4
    tau: float = 0.6
    kn_sensor: int = 1
    newton_tol: float = 1e-12
    newton_maxit: int = 30
    newton_min_upd: int = 0
    rho_inf: float = 1.0
    u_inf: tuple = (0.0, 0.0, 0.0)
    T_inf: float = 0.5
    init_maxit: int = 200
    prandtl: float = 1.0
    root_finder: int = 0

    def params(self) -> Params:
        p = Params()
        p.nx, p.ny, p.nz = self.nx, self.ny, self.nz
        for d in range(3):
            p.periodic[d] = int(self.periodic[d])
            p.u_inf[d] = float(self.u_inf[d])
        p.gamma = self.gamma
        p.tau = self.tau
        p.kn_sensor = int(self.kn_sensor)
        p.newton_tol = self.newton_tol
        p.newton_maxit = int(self.newton_maxit)
        p.newton_min_upd = int(self.newton_min_upd)
        p.rho_inf = self.rho_inf
        p.T_inf = self.T_inf
        p.prandtl = self.prandtl
        p.root_finder = int(self.root_finder)
        return p

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz


def cell_macros(cfg: Config, f, g):
    rho = ctypes.c_double()
    T = ctypes.c_double()
    u = np.zeros(3)
    p = cfg.params()
    lib().o39_cell_macros(ctypes.byref(p), _p(_f64(f)), _p(_f64(g)), ctypes.byref(rho), _p(u),
                          ctypes.byref(T))
    return rho.value, u, T.value


def collide_cell(cfg: Config, f, g, lam, on_fallback: bool = False, t: int = 0):
    """One collision in place on copies; returns (f*, g*, lam, n_upd, eps, alpha, status,
    on_fallback).  on_fallback (the cell's flag) and t (the time step being taken) decide the
    solve's budget under the failure policy (oracle39.c)."""
    f = _f64(f).copy()
    g = _f64(g).copy()
    lam = _f64(lam).copy()
    fb = ctypes.c_uint8(1 if on_fallback else 0)
    nu = ctypes.c_int()
    eps = ctypes.c_double()
    al = ctypes.c_double()
    p = cfg.params()
    st = lib().o39_collide_cell(ctypes.byref(p), _p(f), _p(g), _p(lam), ctypes.byref(fb), int(t),
                                ctypes.byref(nu), ctypes.byref(eps), ctypes.byref(al))
    return f, g, lam, nu.value, eps.value, al.value, st, bool(fb.value)


def equilibrium(cfg: Config, rho, u, T, maxit=200):
    """(feq, geq, lam, status) of the state (rho, u, T) from a cold start."""
    feq = np.zeros(Q)
    geq = np.zeros(Q)
    lam = np.zeros(NM)
    p = cfg.params()
    st = lib().o39_equilibrium(ctypes.byref(p), float(rho), _p(_f64(u)), float(T), _p(feq),
                               _p(geq), _p(lam), int(maxit), None)
    return feq, geq, lam, st


def newton_fp32start(m, lam0, tol=1e-12, maxit=30, min_upd=0):
    """Newton with a single-precision direction after a single-precision start:
    (lam, F, n_updates, n_float_steps, status); n_updates counts the double-precision ones."""
    lam = _f64(lam0).copy()
    F = np.zeros(Q)
    nu = ctypes.c_int(0)
    n32 = ctypes.c_int(0)
    st = lib().o39_newton_fp32start(_p(_f64(m)), _p(lam), float(tol), int(maxit), int(min_upd),
                                    ctypes.byref(nu), ctypes.byref(n32), _p(F))
    return lam, F, nu.value, n32.value, st


# ---------------------------------------------------------------------------
# Lattice-level state.

@dataclass
class State:
    """Oracle lattice state: populations f, g (N, 39), multipliers lam (N, 13), the per-cell
    "on the fallback" flags on_fb (N,) of the failure policy, and the time t."""
    cfg: Config
    mask: np.ndarray
    f: np.ndarray
    g: np.ndarray
    lam: np.ndarray
    t: int = 0
    stats: Stats = field(default_factory=Stats)
    on_fb: np.ndarray = None

    def __post_init__(self):
        if self.on_fb is None:
            self.on_fb = np.zeros(self.lam.shape[0], np.uint8)


def init(cfg: Config, mask, rho, u, T, allow_failed: bool = False) -> State:
    """Equilibrium initial state.  rho, T: (N,), u: (3, N) (x fastest in cell index).
    Cells whose 13-moment solve fails take the fallback equilibrium; that raises unless
    allow_failed (then State.init_failed counts them)."""
    N = cfg.ncells
    mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(N)
    rho = _f64(rho).reshape(N)
    u = _f64(u).reshape(3, N)
    T = _f64(T).reshape(N)
    f = np.zeros((N, Q))
    g = np.zeros((N, Q))
    lam = np.zeros((N, NM))
    on_fb = np.zeros(N, np.uint8)
    p = cfg.params()
    failed = lib().o39_init(ctypes.byref(p), _p(mask), _p(rho), _p(u), _p(T), _p(f), _p(g),
                            _p(lam), _p(on_fb), int(cfg.init_maxit))
    if failed and not allow_failed:
        raise RuntimeError(f"oracle init: {failed} cells failed the Newton solve")
    st = State(cfg, mask, f, g, lam, on_fb=on_fb)
    st.init_failed = int(failed)
    return st


def step(st: State, nsteps: int) -> int:
    p = st.cfg.params()
    st.on_fb = np.ascontiguousarray(st.on_fb, dtype=np.uint8)
    failed = lib().o39_step(ctypes.byref(p), _p(st.mask), _p(st.f), _p(st.g), _p(st.lam),
                            _p(st.on_fb), int(st.t), int(nsteps), ctypes.byref(st.stats))
    st.t += nsteps
    return int(failed)


def stream(cfg: Config, mask, fpost, gpost, feq_inf, geq_inf):
    """Streaming alone on given post-collision arrays (N,39); returns (f, g) of fluid cells
    (other rows zero)."""
    N = cfg.ncells
    mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(N)
    fo = np.zeros((N, Q))
    go = np.zeros((N, Q))
    p = cfg.params()
    lib().o39_stream(ctypes.byref(p), _p(mask), _p(_f64(fpost)), _p(_f64(gpost)),
                     _p(_f64(feq_inf)), _p(_f64(geq_inf)), _p(fo), _p(go))
    return fo, go


def macros(st: State):
    """(rho, u(3,N), T, p) of the current pre-collision state."""
    N = st.cfg.ncells
    rho = np.zeros(N)
    u = np.zeros((3, N))
    T = np.zeros(N)
    pr = np.zeros(N)
    p = st.cfg.params()
    lib().o39_macros(ctypes.byref(p), _p(st.mask), _p(st.f), _p(st.g), _p(rho), _p(u), _p(T),
                     _p(pr))
    return rho, u, T, pr


def conserved(st: State) -> np.ndarray:
    """[mass, momentum x/y/z, total energy] summed over fluid cells."""
    out = np.zeros(5)
    p = st.cfg.params()
    lib().o39_conserved(ctypes.byref(p), _p(st.mask), _p(st.f), _p(st.g), _p(out))
    return out
