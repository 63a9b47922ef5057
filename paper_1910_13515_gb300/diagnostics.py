"""Diagnostics of a run, computed on the host from the library's read-out fields.

surface_cp: the pressure coefficient along the airfoil of the NACA0012 setup (Sec. 4), the
quantity the paper compares with reference data (not available here).
"""
from __future__ import annotations

import numpy as np

from .inputs import M_FLUID, M_SOLID, Setup


def surface_cells(s: Setup) -> np.ndarray:
    """Indices of the fluid cells with a solid neighbour along x or y (the first fluid layer
    around the airfoil), in cell order."""
    m = s.mask.reshape(s.ny, s.nx)
    solid = m == M_SOLID
    near = np.zeros_like(solid)
    near[:, 1:] |= solid[:, :-1]
    near[:, :-1] |= solid[:, 1:]
    near[1:, :] |= solid[:-1, :]
    near[:-1, :] |= solid[1:, :]
    return np.flatnonzero((near & (m == M_FLUID)).reshape(-1))


def surface_cp(s: Setup, rho: np.ndarray, T: np.ndarray):
    """C_p = (p - p_inf) / (rho_inf |u_inf|^2 / 2), p = rho T, on the surface cells of the
    airfoil of setup s (inputs.naca).  Returns (x/C, C_p upper, x/C, C_p lower), each side
    sorted by x/C (upper: cells above the chord line y_c)."""
    cells = surface_cells(s)
    x = (cells % s.nx).astype(np.float64)
    y = (cells // s.nx).astype(np.float64)
    xc = (x - s.extra["x_le"]) / s.extra["chord"]
    q = 0.5 * s.rho_inf * float(np.dot(s.u_inf, s.u_inf))
    cp = (rho[cells] * T[cells] - s.rho_inf * s.T_inf) / q
    up = y > s.extra["y_c"]
    out = []
    for side in (up, ~up):
        order = np.argsort(xc[side], kind="stable")
        out += [xc[side][order], cp[side][order]]
    return tuple(out)
