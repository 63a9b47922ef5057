"""Seeded synthetic inputs: initial fields (rho, u, T), masks and run parameters.

This module builds inputs only.  It holds none of the lattice Boltzmann
arithmetic and imports neither the CUDA library nor the oracle, so both sides
of a parity test start from the same arrays.

Conventions: a lattice is (nx, ny, nz) with x fastest; a scalar field is a
float64 array of shape (N,) with N = nx*ny*nz and cell = x + nx*(y + ny*z);
velocity is (3, N).  Mask codes: 0 fluid, 1 solid (half-way bounce-back),
2 freestream (far-field equilibrium), 3 outflow (zero-gradient copy along x).
Non-periodic axes carry 3 boundary layers at each end (the longest lattice
shift is 3 cells, Sec. 3 of arXiv:1910.13515).

Temperatures are lattice temperatures (p = rho T, c_s = sqrt(gamma T)).  The
13-moment solve exists only inside the moment cone of the 39 velocities, so
every recipe keeps T >= ~0.36 and |u| <= ~1.3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

M_FLUID, M_SOLID, M_FREE, M_OUT = 0, 1, 2, 3
GHOST = 3


@dataclass
class Setup:
    """Everything needed to create, initialise and run one lattice."""
    name: str
    nx: int
    ny: int
    nz: int
    periodic: tuple
    gamma: float
    tau: float
    kn_sensor: int
    mask: np.ndarray          # (N,) uint8
    rho: np.ndarray           # (N,)
    u: np.ndarray             # (3, N)
    T: np.ndarray             # (N,)
    rho_inf: float = 1.0
    u_inf: tuple = (0.0, 0.0, 0.0)
    T_inf: float = 0.5
    steps: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def fluid_cells(self) -> int:
        return int((self.mask == M_FLUID).sum())


def _flat(a3: np.ndarray) -> np.ndarray:
    """(nz, ny, nx) -> (N,) with x fastest."""
    return np.ascontiguousarray(a3, dtype=np.float64).reshape(-1)


# ---------------------------------------------------------------------------
# Sod-type Riemann tube.

def riemann_tube(nx: int = 400, rho_l: float = 1.0, p_l: float = 1.0, rho_r: float = 0.125,
                 p_r: float = 0.1, gamma: float = 1.4, tau: float = 0.5, kn_sensor: int = 1,
                 t_scale: float = 0.5, steps: int = 500, x0: float | None = None) -> Setup:
    """1-D Riemann problem along x (ny = nz = 1, periodic y/z, outflow x-ends).

    States are given in normalised units (rho, p) at rest; the lattice
    temperature is T = t_scale * p / rho, so lattice p = rho T = t_scale * p.
    The interface sits between cells nx/2 - 1 and nx/2 unless x0 is given.
    The 3 cells at each x-end are outflow boundary cells.
    """
    x = np.arange(nx, dtype=np.float64)
    xi = (nx / 2 - 0.5) if x0 is None else x0
    left = x < xi
    rho = np.where(left, rho_l, rho_r)
    T = t_scale * np.where(left, p_l / rho_l, p_r / rho_r)
    u = np.zeros((3, nx))
    mask = np.zeros(nx, np.uint8)
    mask[:GHOST] = M_OUT
    mask[nx - GHOST:] = M_OUT
    return Setup(name=f"riemann_{nx}", nx=nx, ny=1, nz=1, periodic=(0, 1, 1), gamma=gamma,
                 tau=tau, kn_sensor=kn_sensor, mask=mask, rho=rho, u=u, T=T,
                 rho_inf=rho_l, u_inf=(0.0, 0.0, 0.0), T_inf=float(T[0]), steps=steps,
                 extra=dict(rho_l=rho_l, p_l=t_scale * p_l, rho_r=rho_r, p_r=t_scale * p_r,
                            x_interface=xi))


def sod(nx: int = 400, **kw) -> Setup:
    """Sod tube: (rho, p) = (1, 1) | (0.125, 0.1), gamma 1.4, at rest; T = p/(2 rho)."""
    return riemann_tube(nx, 1.0, 1.0, 0.125, 0.1, **kw)


# ---------------------------------------------------------------------------
# NACA0012 in supersonic flow (quasi-2-D, nz = 1).

def naca0012_half_thickness(xc: np.ndarray, t: float = 0.12) -> np.ndarray:
    """Analytic NACA 4-digit symmetric half-thickness (open trailing edge), in chords."""
    xc = np.clip(xc, 0.0, 1.0)
    return 5.0 * t * (0.2969 * np.sqrt(xc) - 0.1260 * xc - 0.3516 * xc**2
                      + 0.2843 * xc**3 - 0.1015 * xc**4)


def naca(nx: int = 2048, ny: int = 1024, chord: int = 400, mach: float = 1.5,
         reynolds: float = 1e4, T_inf: float = 0.5, rho_inf: float = 1.0, gamma: float = 1.4,
         x_le: float | None = None, steps: int = 20000) -> Setup:
    """Supersonic flow past a NACA0012 at zero incidence, staircase solid mask.

    Freestream cells on the left, bottom and top (3 layers, corners included),
    outflow cells on the right (3 layers), periodic z with nz = 1.  The leading
    edge is at x = x_le (default nx/4) and y = ny/2 - 0.5 (between two rows).
    u_inf = Ma sqrt(gamma T_inf); tau = 1/2 + u_inf C / (Re T_inf) from
    nu = (tau - 1/2) T.  Initial field: uniform freestream (impulsive start).
    """
    if x_le is None:
        x_le = nx / 4
    yc = ny / 2 - 0.5
    u_inf = mach * math.sqrt(gamma * T_inf)
    tau = 0.5 + u_inf * chord / (reynolds * T_inf)
    X, Y = np.meshgrid(np.arange(nx, dtype=np.float64), np.arange(ny, dtype=np.float64))
    xc = (X - x_le) / chord
    inside = (xc >= 0.0) & (xc <= 1.0) & (np.abs(Y - yc) <= chord * naca0012_half_thickness(xc))
    mask2 = np.zeros((ny, nx), np.uint8)
    mask2[inside] = M_SOLID
    mask2[:, nx - GHOST:] = M_OUT
    mask2[:, :GHOST] = M_FREE
    mask2[:GHOST, :] = M_FREE
    mask2[ny - GHOST:, :] = M_FREE
    N = nx * ny
    rho = np.full(N, rho_inf)
    u = np.zeros((3, N))
    u[0, :] = u_inf
    T = np.full(N, T_inf)
    return Setup(name=f"naca0012_{nx}x{ny}_C{chord}", nx=nx, ny=ny, nz=1, periodic=(0, 0, 1),
                 gamma=gamma, tau=tau, kn_sensor=1, mask=mask2.reshape(-1), rho=rho, u=u, T=T,
                 rho_inf=rho_inf, u_inf=(u_inf, 0.0, 0.0), T_inf=T_inf, steps=steps,
                 extra=dict(chord=chord, mach=mach, reynolds=reynolds, x_le=x_le, y_c=yc))


# ---------------------------------------------------------------------------
# Periodic box with a random solenoidal velocity field (FP64 and precision form).

def limit_speed(u: np.ndarray, umax: float) -> np.ndarray:
    """Smoothly cap |u| below umax: u * umax tanh(|u|/umax) / |u| (direction kept)."""
    s = np.sqrt((u * u).sum(axis=0))
    fac = np.where(s > 0, umax * np.tanh(s / np.maximum(umax, 1e-300)) / np.maximum(s, 1e-300),
                   1.0)
    return u * fac


def solenoidal_field(n: int, seed: int, kmin: float = 1.0, kmax: float = 4.0,
                     shape: tuple | None = None) -> np.ndarray:
    """Random divergence-free field on a periodic n^3 (or `shape`=(nz,ny,nx)) box:
    Gaussian Fourier modes with kmin <= |k| <= kmax projected onto k.u = 0,
    normalised to unit rms |u|.  Returns (3, nz, ny, nx)."""
    nz, ny, nx = shape if shape is not None else (n, n, n)
    rng = np.random.default_rng(seed)
    kx = np.fft.fftfreq(nx) * nx
    ky = np.fft.fftfreq(ny) * ny
    kz = np.fft.fftfreq(nz) * nz
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    K2 = KX**2 + KY**2 + KZ**2
    band = (K2 >= kmin**2) & (K2 <= kmax**2)
    U = np.zeros((3, nz, ny, nx), np.complex128)
    for d in range(3):
        U[d][band] = rng.standard_normal(band.sum()) + 1j * rng.standard_normal(band.sum())
    kdotu = KX * U[0] + KY * U[1] + KZ * U[2]
    K2s = np.where(K2 > 0, K2, 1.0)
    U[0] -= KX * kdotu / K2s
    U[1] -= KY * kdotu / K2s
    U[2] -= KZ * kdotu / K2s
    u = np.real(np.fft.ifftn(U, axes=(1, 2, 3)))
    rms = math.sqrt(float((u * u).sum(axis=0).mean()))
    return u / rms


def box(n: int = 256, seed: int = 0, mach_rms: float = 0.8, T_mean: float = 0.5,
        noise: float = 0.05, gamma: float = 1.4, tau: float = 0.55, kn_sensor: int = 1,
        umax: float = 1.2, steps: int = 1000, shape: tuple | None = None) -> Setup:
    """Periodic box: solenoidal low-band velocity at rms |u| = mach_rms sqrt(gamma T_mean),
    speeds smoothly capped below umax (the 13-moment solve needs |u| < ~1.5 at T = 0.5),
    rho = 1 + noise U, T = T_mean (1 + noise U'), U, U' ~ uniform[-1, 1) i.i.d. per cell.
    shape=(nz, ny, nx) overrides the cube n^3."""
    nz, ny, nx = shape if shape is not None else (n, n, n)
    u0 = solenoidal_field(n, seed, shape=(nz, ny, nx))
    target = mach_rms * math.sqrt(gamma * T_mean)
    # scale so the capped field has the target rms (bisection on a fixed subsample)
    flat = u0.reshape(3, -1)
    sub = flat[:, np.random.default_rng(seed + 104729).choice(
        flat.shape[1], min(flat.shape[1], 1 << 18), replace=False)]
    lo, hi = 0.0, 4.0 * target
    for _ in range(50):
        mid = 0.5 * (lo + hi)
        uc = limit_speed(mid * sub, umax)
        if math.sqrt(float((uc * uc).sum(axis=0).mean())) < target:
            lo = mid
        else:
            hi = mid
    u = limit_speed(0.5 * (lo + hi) * u0, umax)
    rng = np.random.default_rng(seed + 7919)
    N = nx * ny * nz
    rho = 1.0 + noise * rng.uniform(-1.0, 1.0, N)
    T = T_mean * (1.0 + noise * rng.uniform(-1.0, 1.0, N))
    return Setup(name=f"box_{nx}x{ny}x{nz}_s{seed}", nx=nx, ny=ny, nz=nz, periodic=(1, 1, 1),
                 gamma=gamma, tau=tau, kn_sensor=kn_sensor, mask=np.zeros(N, np.uint8),
                 rho=rho, u=u.reshape(3, N), T=T, rho_inf=1.0, T_inf=T_mean, steps=steps,
                 extra=dict(seed=seed, mach_rms=mach_rms, umax=umax))



def subsonic_box(nx: int, ny: int, nz: int = 1, seed: int = 0, mach_rms: float = 0.3,
                 T_mean: float = 2.0 / 3.0, noise: float = 0.01, gamma: float = 1.4,
                 tau: float = 0.6) -> Setup:
    """Generic subsonic periodic flow for the polynomial-equilibrium comparison model: the
    box() recipe at rms |u| = mach_rms sqrt(gamma T_mean) about the lattice temperature 2/3,
    rho and T with 1 % noise, plain BGK."""
    s = box(seed=seed, shape=(nz, ny, nx), mach_rms=mach_rms, T_mean=T_mean, noise=noise,
            gamma=gamma, tau=tau, kn_sensor=0)
    s.name = f"subsonic_{nx}x{ny}x{nz}_s{seed}"
    return s

def uniform(nx: int, ny: int, nz: int, rho: float = 1.0, u=(0.3, -0.2, 0.1), T: float = 0.5,
            gamma: float = 1.4, tau: float = 0.6, kn_sensor: int = 1) -> Setup:
    """Uniform periodic flow (an invariant of the method)."""
    N = nx * ny * nz
    uu = np.zeros((3, N))
    for d in range(3):
        uu[d] = u[d]
    return Setup(name=f"uniform_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, periodic=(1, 1, 1),
                 gamma=gamma, tau=tau, kn_sensor=kn_sensor, mask=np.zeros(N, np.uint8),
                 rho=np.full(N, rho), u=uu, T=np.full(N, T), rho_inf=rho, u_inf=tuple(u),
                 T_inf=T)


# ---------------------------------------------------------------------------
# Serving-form building blocks: shear layers and random Riemann tubes.

def shear_layer(L: int, mach: float, T_mean: float = 0.7, gamma: float = 1.4, tau: float = 0.55,
                kn_sensor: int = 1, steps: int = 500, seed: int = 0) -> Setup:
    """Doubly periodic L x L x 1 double shear layer: u_x = dU/2 (tanh((y-L/4)/d)
    - tanh((y-3L/4)/d) - 1) with d = L/40, u_y = 0.05 dU sin(2 pi x/L),
    dU = Ma sqrt(gamma T); rho = 1, T = T_mean.  (`seed` only names the setup.)
    T_mean = 0.7 and tau = 0.55 keep the roll-up of Ma <= 2 layers inside the moment cone
    of D3Q39 (at T_mean = 0.5, tau = 0.52 the Ma >= 1.7 layers cool cells below T = 0.36)."""
    dU = mach * math.sqrt(gamma * T_mean)
    d = L / 40.0
    X, Y = np.meshgrid(np.arange(L, dtype=np.float64), np.arange(L, dtype=np.float64))
    ux = 0.5 * dU * (np.tanh((Y - L / 4) / d) - np.tanh((Y - 3 * L / 4) / d) - 1.0)
    uy = 0.05 * dU * np.sin(2 * math.pi * X / L)
    N = L * L
    u = np.zeros((3, N))
    u[0] = ux.reshape(-1)
    u[1] = uy.reshape(-1)
    return Setup(name=f"shear_{L}_Ma{mach:.2f}", nx=L, ny=L, nz=1, periodic=(1, 1, 1),
                 gamma=gamma, tau=tau, kn_sensor=kn_sensor, mask=np.zeros(N, np.uint8),
                 rho=np.ones(N), u=u, T=np.full(N, T_mean), T_inf=T_mean, steps=steps,
                 extra=dict(mach=mach, seed=seed))


def _star_pressure(rl, pl, rr, pr, g):
    """Star-region pressure and velocity of a Riemann problem at rest (used only to
    reject unrealisable random draws; plain Newton on the pressure function)."""
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)

    def fk(p, r, pk, a):
        if p > pk:
            A, B = 2.0 / ((g + 1) * r), (g - 1) / (g + 1) * pk
            return (p - pk) * math.sqrt(A / (p + B))
        return 2 * a / (g - 1) * ((p / pk) ** ((g - 1) / (2 * g)) - 1)

    lo, hi = 1e-12, 10 * max(pl, pr)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if fk(mid, rl, pl, al) + fk(mid, rr, pr, ar) > 0:
            hi = mid
        else:
            lo = mid
    p = 0.5 * (lo + hi)
    u = 0.5 * (fk(p, rr, pr, ar) - fk(p, rl, pl, al))
    return p, u


def random_riemann(rng: np.random.Generator, nmin=200, nmax=4000, gamma=1.4, tau=0.5,
                   steps=None) -> Setup:
    """Random Riemann tube: N ~ U[nmin, nmax], rho_L, rho_R ~ U[0.1, 1], p_L/p_R ~ U[2, 20],
    at rest; redrawn until the initial and star-region lattice temperatures lie in
    [0.4, 0.9] and [0.38, 1.2] and |u*| <= 1.0."""
    g = gamma
    while True:
        n = int(rng.integers(nmin, nmax + 1))
        rl, rr = rng.uniform(0.1, 1.0, 2)
        ratio = rng.uniform(2.0, 20.0)
        Tr = rng.uniform(0.4, 0.9)
        pr = rr * Tr
        pl = ratio * pr
        Tl = pl / rl
        if not (0.4 <= Tl <= 0.9):
            continue
        ps, us = _star_pressure(rl, pl, rr, pr, g)
        Tsl = Tl * (ps / pl) ** ((g - 1) / g)          # isentropic from the left state
        mu = (g - 1) / (g + 1)
        rsr = rr * (ps / pr + mu) / (mu * ps / pr + 1)  # shock-compressed right state
        Tsr = ps / rsr
        if 0.38 <= Tsl <= 1.2 and 0.38 <= Tsr <= 1.2 and abs(us) <= 1.0:
            break
    st = riemann_tube(n, rl, pl, rr, pr, gamma=g, tau=tau, kn_sensor=1, t_scale=1.0,
                      steps=steps if steps is not None else int(rng.integers(200, 2001)))
    st.name = f"riemann_{n}"
    return st


@dataclass
class Request:
    rid: int
    arrival_s: float
    setup: Setup
    cancel_s: float | None = None   # the client withdraws the request at this time (None: never)


def serving_requests(n: int = 64, seed: int = 0, rate_hz: float = 200.0,
                     riemann_range=(200, 4000), shear_sizes=(128, 256, 512, 1024),
                     steps_range=(200, 2000)) -> list:
    """Poisson stream of n requests, half Riemann tubes and half 2-D shear layers
    (L in shear_sizes, Ma ~ U[0.5, 2]), each with steps ~ U[steps_range]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for rid in range(n):
        t += rng.exponential(1.0 / rate_hz)
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        if rng.uniform() < 0.5:
            st = random_riemann(rng, riemann_range[0], riemann_range[1], steps=steps)
        else:
            L = int(rng.choice(shear_sizes))
            st = shear_layer(L, float(rng.uniform(0.5, 2.0)), steps=steps, seed=rid)
        reqs.append(Request(rid, t, st))
    return reqs
