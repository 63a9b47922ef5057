"""Pins of the oracle's Prandtl-number adjustment (Sec. 3 names a quasi-equilibrium
collision and leaves it out; the oracle's reading is a two-relaxation-time quasi-equilibrium
whose heat flux is carried by g): each pin comes from the mathematics, not from the oracle's
formulas -- the moment identities a quasi-equilibrium collision must satisfy, the special
case Pr = 1, and the Chapman-Enskog ratio of the thermal diffusivities measured from the decay
of a temperature wave."""
import math

import numpy as np

from paper_1910_13515_gb300 import inputs

RNG = np.random.default_rng(2024)


def _noneq_cell(oracle, cfg, amp, rng):
    u = rng.uniform(-0.4, 0.4, 3)
    T = rng.uniform(0.45, 0.75)
    rho = rng.uniform(0.5, 1.5)
    feq, geq, lam, st = oracle.equilibrium(cfg, rho, u, T)
    assert st == 0
    f = feq * (1 + amp * rng.uniform(-1, 1, 39))
    g = geq * (1 + amp * rng.uniform(-1, 1, 39))
    return f, g, lam


def _moments(vel, f, g):
    """mass, momentum (3), total energy, the heat flux q (3) about the cell's own velocity,
    and the six second moments of f about that velocity."""
    v = vel.astype(float)
    rho = f.sum()
    u = (f @ v) / rho
    c = v - u
    c2 = (c ** 2).sum(1)
    q = 0.5 * ((c2 * f + g) @ c)
    P = np.array([(f * c[:, a] * c[:, b]).sum() for a, b in
                  ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))])
    e = 0.5 * (f @ (v ** 2).sum(1) + g.sum())
    return rho, rho * u, e, q, P


def test_heat_flux_relaxes_with_tau2_and_the_stress_with_tau(oracle):
    """One collision multiplies the heat flux (about the cell velocity, which the collision
    keeps) by 1 - 1/tau2 with tau2 = 1/2 + (tau - 1/2)/Pr, and the deviation of the stress from
    its equilibrium value rho T I by 1 - 1/tau: the two-relaxation-time property, with the heat
    flux of the 13-moment equilibrium zero."""
    vel, _, _ = oracle.lattice()
    for Pr in (0.71, 2.0, 0.3):
        tau = 0.62
        tau2 = 0.5 + (tau - 0.5) / Pr
        cfg = oracle.Config(nx=1, tau=tau, kn_sensor=0, prandtl=Pr)
        for _ in range(25):
            f, g, lam = _noneq_cell(oracle, cfg, 0.05, RNG)
            rho0, j0, e0, q0, P0 = _moments(vel, f, g)
            fs, gs, lam2, nu, eps, al, st, _ = oracle.collide_cell(cfg, f, g, lam)
            assert st == 0
            rho1, j1, e1, q1, P1 = _moments(vel, fs, gs)
            T = (2 * e0 - (j0 @ j0) / rho0) / ((2 / (cfg.gamma - 1)) * rho0)
            scale = np.abs(q0).max()
            assert np.abs(q1 - (1 - 1 / tau2) * q0).max() <= 1e-12 * max(scale, 1e-3), Pr
            Peq = rho0 * T * np.array([1, 1, 1, 0, 0, 0.0])
            assert np.abs((P1 - Peq) - (1 - 1 / tau) * (P0 - Peq)).max() <= 1e-12


def test_collision_with_the_adjustment_conserves(oracle):
    vel, _, _ = oracle.lattice()
    cfg = oracle.Config(nx=1, tau=0.57, kn_sensor=1, prandtl=0.71)
    for amp in (1e-3, 5e-2, 0.3):
        for _ in range(20):
            f, g, lam = _noneq_cell(oracle, cfg, amp, RNG)
            rho0, j0, e0, _, _ = _moments(vel, f, g)
            fs, gs, *_ = oracle.collide_cell(cfg, f, g, lam)
            rho1, j1, e1, _, _ = _moments(vel, fs, gs)
            tol = 64 * np.finfo(float).eps
            assert abs(rho1 - rho0) <= tol * rho0 * 4
            assert np.abs(j1 - j0).max() <= tol * 30 * rho0
            assert abs(e1 - e0) <= tol * 30 * e0


def test_prandtl_one_is_plain_bgk(oracle):
    """Pr = 1 is the paper's collision bit for bit; Pr = 1 + 1e-9 differs by O(1e-9)."""
    cfg0 = oracle.Config(nx=1, tau=0.6, kn_sensor=1)
    cfg1 = oracle.Config(nx=1, tau=0.6, kn_sensor=1, prandtl=1.0)
    cfgn = oracle.Config(nx=1, tau=0.6, kn_sensor=1, prandtl=1.0 + 1e-9)
    for _ in range(10):
        f, g, lam = _noneq_cell(oracle, cfg0, 0.05, RNG)
        a = oracle.collide_cell(cfg0, f, g, lam)
        b = oracle.collide_cell(cfg1, f, g, lam)
        c = oracle.collide_cell(cfgn, f, g, lam)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert np.array_equal(a[0], c[0])
        d = np.abs(c[1] - a[1]).max() / np.abs(a[1]).max()
        assert 0 < d < 1e-8


def _wave_decay(oracle, field, tau, Pr, L=48, T0=0.5, amp=2e-3, steps=(20, 420)):
    """Decay rate per step of the k = 2 pi / L Fourier mode of a periodic 1-D wave: 'T' is a
    temperature wave at uniform pressure (the entropy mode), 'uy' a transverse shear wave."""
    x = np.arange(L)
    k = 2 * math.pi / L
    s = inputs.uniform(L, 1, 1, u=(0, 0, 0), T=T0, tau=tau, kn_sensor=0)
    s.u, s.T, s.rho = s.u.copy(), s.T.copy(), s.rho.copy()
    if field == "T":
        s.T = T0 * (1 + amp * np.sin(k * x))
        s.rho = T0 / s.T
    else:
        s.u[1] = amp * np.sin(k * x)
    cfg = oracle.Config(nx=L, ny=1, nz=1, gamma=s.gamma, tau=tau, kn_sensor=0, prandtl=Pr)
    st = oracle.init(cfg, s.mask, s.rho, s.u, s.T)
    a = []
    for t in steps:
        oracle.step(st, t - st.t)
        rho, u, T, p = oracle.macros(st)
        a.append(((T - T.mean()) if field == "T" else u[1]) @ np.sin(k * x))
    return -math.log(a[1] / a[0]) / (steps[1] - steps[0]) / (k * k)


def test_thermal_diffusivity_scales_as_the_chapman_enskog_ratio(oracle):
    """The entropy mode decays at the thermal diffusivity, which the quasi-equilibrium sets
    through tau2: chi(Pr) / chi(1) = (tau2 - 1/2)/(tau - 1/2) = 1/Pr; the shear-wave
    viscosity does not depend on Pr."""
    tau = 0.8
    chi1 = _wave_decay(oracle, "T", tau, 1.0)
    nu1 = _wave_decay(oracle, "uy", tau, 1.0)
    for Pr in (0.71, 2.0):
        chi = _wave_decay(oracle, "T", tau, Pr)
        nu = _wave_decay(oracle, "uy", tau, Pr)
        assert abs((chi / chi1) * Pr - 1) < 0.03, (Pr, chi / chi1)
        assert abs(nu / nu1 - 1) < 0.01, (Pr, nu / nu1)
