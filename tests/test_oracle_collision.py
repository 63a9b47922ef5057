"""Pins of the oracle's BGK collision with the Knudsen sensor (Sec. 3 of arXiv:1910.13515)."""
import numpy as np

RNG = np.random.default_rng(99)


def _moments(vel, f, g):
    c2 = (vel.astype(float) ** 2).sum(1)
    return np.array([f.sum(), f @ vel[:, 0], f @ vel[:, 1], f @ vel[:, 2],
                     0.5 * (f @ c2 + g.sum())])


def _noneq_cell(oracle, cfg, amp, rng):
    """A cell near a realizable equilibrium (|u| <= 0.5, T in [0.5, 0.7]), perturbed by up to
    `amp` relative per population (kept inside the moment cone for amp < 1)."""
    u = rng.uniform(-0.3, 0.3, 3)
    T = rng.uniform(0.5, 0.7)
    rho = rng.uniform(0.5, 1.5)
    feq, geq, lam, st = oracle.equilibrium(cfg, rho, u, T)
    f = feq * (1 + amp * rng.uniform(-1, 1, 39))
    g = geq * (1 + amp * rng.uniform(-1, 1, 39))
    return f, g, lam


def test_collision_conserves_mass_momentum_energy(oracle):
    vel, _, _ = oracle.lattice()
    for kn in (0, 1):
        cfg = oracle.Config(nx=1, tau=0.57, kn_sensor=kn)
        for amp in (1e-3, 5e-2, 0.3, 0.9):
            for _ in range(20):
                f, g, lam = _noneq_cell(oracle, cfg, amp, RNG)
                m0 = _moments(vel, f, g)
                fs, gs, lam2, nu, eps, al, st, _ = oracle.collide_cell(cfg, f, g, lam)
                assert st == 0
                m1 = _moments(vel, fs, gs)
                # round-off bound: a few dozen ulps of the summed magnitudes
                scale = _moments(np.abs(vel), np.abs(f), np.abs(g)) + \
                    _moments(np.abs(vel), np.abs(fs), np.abs(gs))
                assert np.all(np.abs(m1 - m0) <= 32 * np.finfo(float).eps * scale), \
                    (amp, m1 - m0)


def test_equilibrium_is_a_fixed_point(oracle):
    cfg = oracle.Config(nx=1, tau=0.6)
    for _ in range(20):
        u = RNG.uniform(-0.4, 0.4, 3)
        T = RNG.uniform(0.45, 0.8)
        feq, geq, lam, st = oracle.equilibrium(cfg, 1.3, u, T)
        fs, gs, lam2, nu, eps, al, st, _ = oracle.collide_cell(cfg, feq, geq, lam)
        assert eps < 1e-12 and al == 1.0
        assert np.allclose(fs, feq, rtol=1e-12, atol=0)
        assert np.allclose(gs, geq, rtol=1e-12, atol=0)


def test_bgk_relaxation_and_sensor(oracle):
    """h* = h - (h - h^eq)/(tau alpha(eps)), eps = mean_i |f_i - f_i^eq| / f_i^eq (f only)."""
    vel, _, _ = oracle.lattice()
    tau = 0.57
    for amp, kn in ((0.004, 1), (0.05, 1), (0.5, 1), (0.95, 1), (0.5, 0)):
        cfg = oracle.Config(nx=1, tau=tau, kn_sensor=kn)
        f, g, lam = _noneq_cell(oracle, cfg, amp, RNG)
        fs, gs, lam2, nu, eps, al, st, _ = oracle.collide_cell(cfg, f, g, lam)
        rho, u, T = oracle.cell_macros(cfg, f, g)
        feq, geq, _, _ = oracle.equilibrium(cfg, rho, u, T)
        eps_ref = np.mean(np.abs(f - feq) / feq)
        assert abs(eps - eps_ref) <= 1e-10 * max(eps_ref, 1e-3)
        if kn:
            want = 1.0 if eps_ref < 1e-2 else 1.05 if eps_ref < 1e-1 else 1.35 if eps_ref < 1 \
                else 1.0 / tau
        else:
            want = 1.0
        assert al == want
        te = tau * want
        assert np.allclose(fs, f - (f - feq) / te, rtol=1e-11, atol=1e-15)
        assert np.allclose(gs, g - (g - geq) / te, rtol=1e-11, atol=1e-15)


def test_large_knudsen_number_resets_to_equilibrium(oracle):
    """eps >= 1 gives alpha = 1/tau, tau_eff = 1: the populations become h^eq."""
    cfg = oracle.Config(nx=1, tau=0.52, kn_sensor=1)
    f, g, lam = _noneq_cell(oracle, cfg, 0.9, RNG)
    f[::2] *= 4.0  # strongly non-equilibrium but positive
    fs, gs, lam2, nu, eps, al, st, _ = oracle.collide_cell(cfg, f, g, lam)
    assert eps >= 1.0 and al == 1.0 / 0.52
    rho, u, T = oracle.cell_macros(cfg, f, g)
    feq, geq, _, _ = oracle.equilibrium(cfg, rho, u, T)
    assert np.allclose(fs, feq, rtol=1e-11)
    assert np.allclose(gs, geq, rtol=1e-11)


def test_macros_invert_the_equilibrium(oracle):
    for gamma in (1.4, 1.6):
        cfg = oracle.Config(nx=1, gamma=gamma)
        u = np.array([0.3, -0.6, 0.1])
        feq, geq, lam, st = oracle.equilibrium(cfg, 0.8, u, 0.55)
        rho, uu, T = oracle.cell_macros(cfg, feq, geq)
        assert abs(rho - 0.8) < 1e-14 and np.allclose(uu, u, atol=1e-14) and abs(T - 0.55) < 1e-13
