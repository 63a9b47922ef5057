"""Plain FP64 CPU oracle of the paper's comparison model: BGK with a fourth-order
polynomial equilibrium on the D3Q39 lattice, with a second population set g that
carries the energy of the extra degrees of freedom, so that gamma is free (Sec. 5,
Implementation and efficiency; the double-population approach of Sec. 3).

TEST INFRASTRUCTURE ONLY: the test suite and the CPU-baseline leg of ``bench.py``
are the only callers.  The CUDA library never imports this module and this module
never imports the CUDA library.

The paper names this model but prints no formula for it.  Readings:

- The equilibrium is the Hermite expansion of the Maxwell-Boltzmann distribution
  (mean u, temperature T) about the lattice reference temperature theta0 = 2/3
  (the second moment of the D3Q39 weights per axis), truncated after the fourth
  order ("fourth order in the Mach number"), every temperature term kept:

      f_i^eq = w_i sum_{n=0..4} a^(n) : H^(n)(xi_i) / (n! theta0^n),

  with H^(n) the tensor Hermite polynomials of variance theta0 and a^(n) the
  Hermite coefficients of the Maxwellian, a^(n) = int f^MB H^(n) dxi.
- g_i^eq = (2 C_v - D) T f_i^eq, the double population of the 13-moment model.
- rho, u and T from the populations as in the 13-moment model (T from the total
  energy sum f|xi|^2 + sum g = rho u^2 + 2 C_v rho T).
- Plain BGK with one relaxation time for f and g; periodic lattices (the paper
  times this model on a generic subsonic flow).

Every array of populations is (N, 39) with the cell index x fastest.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import oracle39

Q = 39
D = 3
THETA0 = 2.0 / 3.0


def lattice():
    """D3Q39 velocities (39, 3) float and weights (39,), from the exponential-model oracle."""
    vel, w, _ = oracle39.lattice()
    return vel.astype(np.float64), w


def _sym_pairs(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """The six index placements of a rank-2 tensor a and a rank-2 tensor b in a
    rank-4 tensor: a_ij b_kl + a_ik b_jl + a_il b_jk + a_jk b_il + a_jl b_ik + a_kl b_ij.
    a, b: (..., 3, 3)."""
    return (np.einsum("...ij,...kl->...ijkl", a, b) + np.einsum("...ik,...jl->...ijkl", a, b)
            + np.einsum("...il,...jk->...ijkl", a, b) + np.einsum("...jk,...il->...ijkl", a, b)
            + np.einsum("...jl,...ik->...ijkl", a, b) + np.einsum("...kl,...ij->...ijkl", a, b))


def _delta_delta() -> np.ndarray:
    """d_ij d_kl + d_ik d_jl + d_il d_jk."""
    d = np.eye(D)
    return (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d)
            + np.einsum("il,jk->ijkl", d, d))


def _vec_delta(v: np.ndarray) -> np.ndarray:
    """v_i d_jk + v_j d_ik + v_k d_ij.  v: (..., 3) -> (..., 3, 3, 3)."""
    d = np.eye(D)
    return (np.einsum("...i,jk->...ijk", v, d) + np.einsum("...j,ik->...ijk", v, d)
            + np.einsum("...k,ij->...ijk", v, d))


def hermite(xi: np.ndarray, theta: float = THETA0):
    """Tensor Hermite polynomials H^(0..4) of variance theta at velocities xi (M, 3):
    H0 = 1, H1 = xi, H2 = xi xi - theta d, H3 = xi xi xi - theta (xi d)_3,
    H4 = xi xi xi xi - theta (xi xi d)_6 + theta^2 (d d)_3 (Grad's polynomials)."""
    xi = np.asarray(xi, dtype=np.float64)
    d = np.eye(D)
    xx = np.einsum("mi,mj->mij", xi, xi)
    H0 = np.ones(len(xi))
    H1 = xi
    H2 = xx - theta * d
    H3 = np.einsum("mij,mk->mijk", xx, xi) - theta * _vec_delta(xi)
    dm = np.broadcast_to(d, xx.shape)
    H4 = (np.einsum("mij,mkl->mijkl", xx, xx) - theta * _sym_pairs(xx, dm)
          + theta**2 * _delta_delta())
    return H0, H1, H2, H3, H4


def mb_coefficients(rho, u, T, theta: float = THETA0):
    """Hermite coefficients a^(0..4) of the Maxwellian rho N(u, T I) in the basis of
    variance theta (closed forms; pinned against the integral in the tests):
    a0 = rho, a1 = rho u, a2 = rho (u u + s d), a3 = rho (u u u + s (u d)_3),
    a4 = rho (u u u u + s (u u d)_6 + s^2 (d d)_3), s = T - theta.
    rho, T: (N,); u: (N, 3)."""
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    s = np.asarray(T, dtype=np.float64) - theta
    d = np.eye(D)
    uu = np.einsum("ni,nj->nij", u, u)
    a0 = rho
    a1 = rho[:, None] * u
    a2 = rho[:, None, None] * (uu + s[:, None, None] * d)
    a3 = rho[:, None, None, None] * (np.einsum("nij,nk->nijk", uu, u)
                                     + s[:, None, None, None] * _vec_delta(u))
    dn = np.broadcast_to(d, uu.shape)
    a4 = rho[:, None, None, None, None] * (
        np.einsum("nij,nkl->nijkl", uu, uu) + s[:, None, None, None, None] * _sym_pairs(uu, dn)
        + (s**2)[:, None, None, None, None] * _delta_delta())
    return a0, a1, a2, a3, a4


def expansion(xi, rho, u, T, theta: float = THETA0) -> np.ndarray:
    """sum_{n<=4} a^(n) : H^(n)(xi) / (n! theta^n) for each cell (N) and velocity (M):
    the polynomial that multiplies the weight (lattice) or the Gaussian (continuum).
    Returns (N, M)."""
    H = hermite(xi, theta)
    a = mb_coefficients(np.atleast_1d(rho), np.atleast_2d(u), np.atleast_1d(T), theta)
    out = a[0][:, None] * H[0][None, :]
    out = out + np.einsum("ni,mi->nm", a[1], H[1]) / theta
    out = out + np.einsum("nij,mij->nm", a[2], H[2]) / (2.0 * theta**2)
    out = out + np.einsum("nijk,mijk->nm", a[3], H[3]) / (6.0 * theta**3)
    out = out + np.einsum("nijkl,mijkl->nm", a[4], H[4]) / (24.0 * theta**4)
    return out


def feq(rho, u, T) -> np.ndarray:
    """f_i^eq = w_i * expansion(xi_i) on D3Q39: (N, 39)."""
    vel, w = lattice()
    return w[None, :] * expansion(vel, rho, u, T)


@dataclass
class Config:
    nx: int
    ny: int = 1
    nz: int = 1
    gamma: float = 1.4
    tau: float = 0.6

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def cg(self) -> float:
        """2 C_v - D: the weight of T f^eq in g^eq."""
        return 2.0 / (self.gamma - 1.0) - D


def equilibrium(cfg: Config, rho, u, T):
    """(f^eq, g^eq), each (N, 39), of cells with rho (N,), u (3, N), T (N,)."""
    rho = np.asarray(rho, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    f = feq(rho, np.asarray(u, dtype=np.float64).T, T)
    return f, cfg.cg * T[:, None] * f


def macros(cfg: Config, f, g):
    """rho (N,), u (3, N), T (N,) of populations f, g (N, 39):
    rho = sum f, rho u = sum f xi, T = (sum f|xi|^2 + sum g - rho u^2) / (2 C_v rho)."""
    vel, _ = lattice()
    rho = f.sum(axis=1)
    u = (f @ vel).T / rho
    e2 = f @ (vel**2).sum(axis=1) + g.sum(axis=1)
    cv = 1.0 / (cfg.gamma - 1.0)
    T = (e2 - rho * (u**2).sum(axis=0)) / (2.0 * cv * rho)
    return rho, u, T


def collide(cfg: Config, f, g):
    """BGK: h* = h - (h - h^eq) / tau for f and g."""
    rho, u, T = macros(cfg, f, g)
    fe, ge = equilibrium(cfg, rho, u, T)
    om = 1.0 / cfg.tau
    return f - om * (f - fe), g - om * (g - ge)


def stream(cfg: Config, h) -> np.ndarray:
    """Periodic pull streaming h_i(x, t+1) = h*_i(x - xi_i, t) of (N, 39) arrays."""
    vel, _ = lattice()
    grid = h.reshape(cfg.nz, cfg.ny, cfg.nx, Q)
    out = np.empty_like(grid)
    for i in range(Q):
        cx, cy, cz = (int(c) for c in vel[i])
        out[..., i] = np.roll(grid[..., i], shift=(cz, cy, cx), axis=(0, 1, 2))
    return out.reshape(cfg.ncells, Q)


@dataclass
class State:
    cfg: Config
    f: np.ndarray
    g: np.ndarray
    t: int = 0


def init(cfg: Config, rho, u, T) -> State:
    f, g = equilibrium(cfg, rho, u, T)
    return State(cfg=cfg, f=f, g=g, t=0)


def step(st: State, nsteps: int) -> None:
    """nsteps of collide-then-stream."""
    for _ in range(nsteps):
        fs, gs = collide(st.cfg, st.f, st.g)
        st.f = stream(st.cfg, fs)
        st.g = stream(st.cfg, gs)
        st.t += 1


def conserved(st: State) -> np.ndarray:
    """[mass, momentum x/y/z, total energy] = sums of rho, rho u, (sum f|xi|^2 + sum g)/2."""
    vel, _ = lattice()
    mass = st.f.sum()
    mom = (st.f @ vel).sum(axis=0)
    energy = 0.5 * ((st.f @ (vel**2).sum(axis=1)).sum() + st.g.sum())
    return np.array([mass, mom[0], mom[1], mom[2], energy])

