"""Exact solution of the 1-D Riemann problem for an ideal gas (Euler equations).

TEST INFRASTRUCTURE ONLY (a pin for the Sod tube of Sec. 4 of arXiv:1910.13515,
which compares the lattice Boltzmann tube against the theoretical solution).

Standard construction: the star-region pressure p* solves
f_L(p*) + f_R(p*) + (u_R - u_L) = 0, where f_K is the shock (Rankine-Hugoniot)
branch for p > p_K and the rarefaction (isentropic, Riemann invariant) branch
otherwise; u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2.  The similarity
solution is then sampled at xi = (x - x0)/t.
"""
from __future__ import annotations

import math

import numpy as np


def _fk(p, rk, pk, ak, g):
    """Pressure function of one side and its derivative."""
    if p > pk:
        A = 2.0 / ((g + 1.0) * rk)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    e = (g - 1.0) / (2.0 * g)
    return (2.0 * ak / (g - 1.0)) * ((p / pk) ** e - 1.0), (1.0 / (rk * ak)) * (p / pk) ** (-(g + 1.0) / (2.0 * g))


def star_state(rl, ul, pl, rr, ur, pr, g=1.4, tol=1e-15, maxit=100):
    """(p*, u*) by Newton on the pressure function from the two-rarefaction guess."""
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    du = ur - ul
    if 2.0 * (al + ar) / (g - 1.0) <= du:
        raise ValueError("vacuum generated")
    e = (g - 1.0) / (2.0 * g)
    p = ((al + ar - 0.5 * (g - 1.0) * du) / (al / pl**e + ar / pr**e)) ** (1.0 / e)
    for _ in range(maxit):
        fl, dl = _fk(p, rl, pl, al, g)
        fr, dr = _fk(p, rr, pr, ar, g)
        pn = p - (fl + fr + du) / (dl + dr)
        if pn <= 0:
            pn = 0.5 * p
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, al, g)
    fr, _ = _fk(p, rr, pr, ar, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(xi, rl, ul, pl, rr, ur, pr, g=1.4):
    """(rho, u, p) arrays at similarity coordinates xi = x/t."""
    ps, us = star_state(rl, ul, pl, rr, ur, pr, g)
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    mu = (g - 1.0) / (g + 1.0)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for n, s in enumerate(xi.flat):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                S = ul - al * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s < S:
                    r, v, q = rl, ul, pl
                else:
                    r, v, q = rl * (ps / pl + mu) / (mu * ps / pl + 1.0), us, ps
            else:  # left rarefaction
                head = ul - al
                asl = al * (ps / pl) ** ((g - 1) / (2 * g))
                tail = us - asl
                if s < head:
                    r, v, q = rl, ul, pl
                elif s > tail:
                    r, v, q = rl * (ps / pl) ** (1 / g), us, ps
                else:
                    c = 2 / (g + 1) + mu / al * (ul - s)
                    r = rl * c ** (2 / (g - 1))
                    v = 2 / (g + 1) * (al + 0.5 * (g - 1) * ul + s)
                    q = pl * c ** (2 * g / (g - 1))
        else:  # right of the contact
            if ps > pr:  # right shock
                S = ur + ar * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s > S:
                    r, v, q = rr, ur, pr
                else:
                    r, v, q = rr * (ps / pr + mu) / (mu * ps / pr + 1.0), us, ps
            else:  # right rarefaction
                head = ur + ar
                asr = ar * (ps / pr) ** ((g - 1) / (2 * g))
                tail = us + asr
                if s > head:
                    r, v, q = rr, ur, pr
                elif s < tail:
                    r, v, q = rr * (ps / pr) ** (1 / g), us, ps
                else:
                    c = 2 / (g + 1) - mu / ar * (ur - s)
                    r = rr * c ** (2 / (g - 1))
                    v = 2 / (g + 1) * (-ar + 0.5 * (g - 1) * ur + s)
                    q = pr * c ** (2 * g / (g - 1))
        rho.flat[n], u.flat[n], p.flat[n] = r, v, q
    return rho, u, p


def shock_speed(rl, ul, pl, rr, ur, pr, g=1.4):
    """Speed of the right-moving shock (requires p* > p_R)."""
    ps, _ = star_state(rl, ul, pl, rr, ur, pr, g)
    ar = math.sqrt(g * pr / rr)
    return ur + ar * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
