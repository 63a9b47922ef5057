"""Whole-step pins of the oracle: invariants, the exact Riemann solution (Sec. 4 of
arXiv:1910.13515) and the transport coefficients of the BGK model."""
import math

import numpy as np
import pytest

from oracle import riemann
from paper_1910_13515_gb300 import inputs


def cfg_of(oracle, s, **kw):
    return oracle.Config(nx=s.nx, ny=s.ny, nz=s.nz, periodic=s.periodic, gamma=s.gamma,
                         tau=s.tau, kn_sensor=s.kn_sensor, rho_inf=s.rho_inf, u_inf=s.u_inf,
                         T_inf=s.T_inf, **kw)


def test_uniform_flow_is_invariant(oracle):
    s = inputs.uniform(4, 3, 2, u=(0.3, -0.2, 0.1), T=0.5)
    st = oracle.init(cfg_of(oracle, s), s.mask, s.rho, s.u, s.T)
    assert oracle.step(st, 300) == 0
    rho, u, T, p = oracle.macros(st)
    assert np.abs(rho - 1).max() < 1e-13
    assert np.abs(u[0] - 0.3).max() < 1e-13 and np.abs(u[1] + 0.2).max() < 1e-13
    assert np.abs(T - 0.5).max() < 1e-13
    assert np.allclose(p, rho * T, rtol=1e-15)


def test_periodic_box_conserves_to_round_off(oracle):
    s = inputs.box(n=8, seed=3, steps=0)
    st = oracle.init(cfg_of(oracle, s), s.mask, s.rho, s.u, s.T)
    c0 = oracle.conserved(st)
    assert oracle.step(st, 30) == 0
    c1 = oracle.conserved(st)
    scale = np.array([c0[0]] * 4 + [c0[4]])
    assert np.all(np.abs(c1 - c0) <= 1e-13 * scale), c1 - c0


def sod_l1(oracle, n):
    s = inputs.sod(n)
    st = oracle.init(cfg_of(oracle, s), s.mask, s.rho, s.u, s.T)
    nstar = int(round(0.3 * n))
    assert oracle.step(st, nstar) == 0
    rho, u, T, p = oracle.macros(st)
    x = np.arange(n, dtype=float)
    e = s.extra
    re, ue, pe = riemann.sample((x - e["x_interface"]) / nstar, e["rho_l"], 0.0, e["p_l"],
                                e["rho_r"], 0.0, e["p_r"], s.gamma)
    fl = s.mask == 0
    return np.abs(rho[fl] - re[fl]).mean(), np.abs(u[0][fl] - ue[fl]).mean(), \
        np.abs(p[fl] - pe[fl]).mean()


def test_sod_converges_to_exact_riemann_solution(oracle):
    """Sod tube, tau = 1/2 with alpha(eps) (the paper's BGK(eps) zero-viscosity case): the L1
    error in rho against the exact solution at t = 0.3 N decreases with N, order >= 0.5."""
    ns = (200, 400, 800)
    errs = [sod_l1(oracle, n) for n in ns]
    erho = [e[0] for e in errs]
    assert erho[0] > erho[1] > erho[2], erho
    order = math.log(erho[0] / erho[2], 2) / math.log(ns[2] / ns[0], 2)
    assert order >= 0.5, (erho, order)
    assert erho[1] < 0.01 and errs[1][1] < 0.01 and errs[1][2] < 0.01, errs


def test_plain_bgk_sod_is_stable_at_tau_057(oracle):
    """The paper's plain-BGK case: tau_f = 0.57 without the sensor stays stable on 400 cells."""
    s = inputs.sod(400, tau=0.57, kn_sensor=0)
    st = oracle.init(cfg_of(oracle, s), s.mask, s.rho, s.u, s.T)
    assert oracle.step(st, 120) == 0
    rho, u, T, p = oracle.macros(st)
    fl = s.mask == 0
    assert np.isfinite(rho[fl]).all() and rho[fl].min() > 0.1 and rho[fl].max() < 1.1


def test_sound_speed(oracle):
    """A standing acoustic wave oscillates with c_s = sqrt(gamma T) (p = rho T)."""
    L, T0, gamma = 48, 0.5, 1.4
    x = np.arange(L)
    k = 2 * np.pi / L
    s = inputs.uniform(L, 1, 1, u=(0, 0, 0), T=T0, gamma=gamma, tau=0.52, kn_sensor=0)
    s.rho = 1 + 1e-4 * np.cos(k * x)
    s.T = T0 * s.rho ** (gamma - 1)  # isentropic perturbation
    st = oracle.init(cfg_of(oracle, s), s.mask, s.rho, s.u, s.T)
    amps = []
    for t in range(90):
        rho, u, T, p = oracle.macros(st)
        amps.append(((rho - 1) * np.cos(k * x)).sum())
        oracle.step(st, 1)
    amps = np.array(amps)
    # first downward zero crossing at a quarter period
    i = np.where((amps[:-1] > 0) & (amps[1:] <= 0))[0][0]
    tq = i + amps[i] / (amps[i] - amps[i + 1])
    c = (L / 4) / tq
    assert abs(c / math.sqrt(gamma * T0) - 1) < 0.02, (c, math.sqrt(gamma * T0))


def test_shear_wave_viscosity(oracle):
    """A transverse shear wave u_y(x) decays at exp(-nu k^2 t).  Chapman-Enskog for BGK gives
    nu = (tau - 1/2) dM3_xxy/du_y of the equilibrium; a Maxwellian has dM3_xxy/du_y = T, but
    the 13-moment equilibrium constrains only the contracted third moment (Eq. 13constraints),
    so on D3Q39 its response is ~0.85 T.  The decay measured from the full step must match the
    response measured from the equilibrium alone (two independent routes)."""
    L, T0, tau = 32, 0.5, 0.8
    x = np.arange(L)
    k = 2 * np.pi / L
    s = inputs.uniform(L, 1, 1, u=(0, 0, 0), T=T0, tau=tau, kn_sensor=0)
    s.u[1] = 1e-3 * np.sin(k * x)
    st = oracle.init(cfg_of(oracle, s), s.mask, s.rho, s.u, s.T)
    a0 = None
    n = 100
    for t in (10, n + 10):
        oracle.step(st, t - st.t)
        rho, u, T, p = oracle.macros(st)
        a = (u[1] * np.sin(k * x)).sum()
        if a0 is None:
            a0 = a
    nu = -math.log(a / a0) / (k * k * n)
    vel, _, _ = oracle.lattice()
    d = 1e-6
    lam, F, _, _ = oracle.newton(oracle.targets([0, d, 0], T0),
                                 oracle.gaussian_guess([0, d, 0], T0), maxit=100)
    c3 = (F * vel[:, 0] ** 2 * vel[:, 1]).sum() / d
    assert 0.8 * T0 < c3 < 0.9 * T0
    assert abs(nu / ((tau - 0.5) * c3) - 1) < 0.03, (nu, (tau - 0.5) * c3)


def test_sod_500_steps_is_roundoff_sensitive(oracle):
    """Documents why the 500-step Sod run is compared statistically: the oracle's own run
    from an initial state perturbed by 1e-15 agrees to 1e-11 at step 160 but not at step 500."""
    from gpu_helpers import rel_diffs
    s = inputs.sod(400)
    a = oracle.init(cfg_of(oracle, s), s.mask, s.rho, s.u, s.T)
    b = oracle.init(cfg_of(oracle, s), s.mask, s.rho, s.u, s.T)
    b.f *= 1 + 1e-15 * np.random.default_rng(0).uniform(-1, 1, b.f.shape)
    oracle.step(a, 160)
    oracle.step(b, 160)
    assert max(rel_diffs(oracle.macros(a), oracle.macros(b), s.mask, s.gamma)) < 1e-11
    oracle.step(a, 340)
    oracle.step(b, 340)
    assert max(rel_diffs(oracle.macros(a), oracle.macros(b), s.mask, s.gamma)) > 1e-6


def test_obstacle_conserves_mass_and_energy_not_momentum(oracle):
    """Half-way bounce-back (Sec. 4) sends each population back to its cell with the same
    speed: on a periodic lattice with a solid block the total mass and energy stay constant
    to round-off, while the momentum changes by the force on the block."""
    s = inputs.box(seed=6, shape=(7, 10, 12))
    m = s.mask.reshape(7, 10, 12)
    m[2:4, 3:6, [10, 11, 0]] = 1
    st = oracle.init(cfg_of(oracle, s), s.mask, s.rho, s.u, s.T)
    c0 = oracle.conserved(st)
    assert oracle.step(st, 101) == 0
    c1 = oracle.conserved(st)
    assert abs(c1[0] - c0[0]) <= 1e-13 * c0[0] and abs(c1[4] - c0[4]) <= 1e-13 * c0[4]
    assert np.abs(c1[1:4] - c0[1:4]).max() > 1e-4 * c0[0]


def test_knudsen_sensor_stabilises_the_airfoil_start(oracle):
    """Sec. 4: on the impulsive Ma 1.5, Re 1e4 airfoil start, plain BGK at tau = 0.506 blows up
    (here within 20 steps at C = 24), while the same run with the Knudsen-number-dependent
    relaxation time (Eq. alpha) stays bounded with every cell inside the moment cone."""
    base = inputs.naca(nx=96, ny=48, chord=24, x_le=24)
    fl = base.mask == 0
    for kn, steps in ((0, 40), (1, 200)):
        base.kn_sensor = kn
        st = oracle.init(cfg_of(oracle, base), base.mask, base.rho, base.u, base.T)
        blew_up = False
        for _ in range(steps // 20):
            oracle.step(st, 20)
            rho, u, T, p = oracle.macros(st)
            with np.errstate(invalid="ignore"):
                if not (np.isfinite(rho[fl]).all() and np.isfinite(T[fl]).all()
                        and (T[fl] > 0).all()):
                    blew_up = True
                    break
        if kn == 0:
            assert blew_up
        else:
            assert not blew_up and st.stats.failed_cells == 0
            assert T[fl].min() > 0.3 and 0.3 < rho[fl].min() and rho[fl].max() < 3.0
