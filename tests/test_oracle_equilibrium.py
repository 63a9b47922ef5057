"""Pins of the oracle's 13-moment equilibrium and Newton solve (Sec. 2, Sec. 3, Sec. 5 of
arXiv:1910.13515) against closed forms and mathematics independent of the oracle."""
import numpy as np
import pytest
from numpy.polynomial.hermite import hermgauss

RNG = np.random.default_rng(1234)


def mb_moment(rho, u, T, p, q, r):
    """int xi_x^p xi_y^q xi_z^r f_MB d^3xi by tensor Gauss-Hermite quadrature (exact for
    these polynomial degrees): f_MB = rho (2 pi T)^(-3/2) exp(-(xi-u)^2/(2T)) (Eq. 1, with the
    minus sign of the Maxwellian)."""
    x, w = hermgauss(12)
    s = np.sqrt(2.0 * T)
    vals = []
    for d, k in enumerate((p, q, r)):
        vals.append(((u[d] + s * x) ** k * w).sum() / np.sqrt(np.pi))
    return rho * vals[0] * vals[1] * vals[2]


MONOS = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2),
         (1, 1, 0), (1, 0, 1), (0, 1, 1)]


def mb_targets(u, T):
    """The 13 Maxwell-Boltzmann moments of Eq. (13constraints), per unit density, by quadrature:
    the 10 monomials of degree <= 2 and the contracted third moments sum_b <xi_a xi_b xi_b>."""
    out = [mb_moment(1.0, u, T, *m) for m in MONOS]
    for a in range(3):
        tot = 0.0
        for b in range(3):
            e = [0, 0, 0]
            e[a] += 1
            e[b] += 2
            tot += mb_moment(1.0, u, T, *e)
        out.append(tot)
    return np.array(out)


def random_state(rng):
    T = rng.uniform(0.4, 0.8)
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    u = d * rng.uniform(0.0, 1.0)
    return u, T


def test_targets_are_maxwell_boltzmann_moments(oracle):
    for _ in range(50):
        u, T = random_state(RNG)
        assert np.allclose(oracle.targets(u, T), mb_targets(u, T), rtol=1e-13, atol=1e-13)


def test_equilibrium_reproduces_13_mb_moments(oracle):
    """Newton from the Gaussian cold start: the discrete equilibrium's 13 moments equal the
    continuous Maxwell-Boltzmann ones to <= 1e-12 relative, relative to max(|M_k|, rho) (the
    density sets the scale of every moment; the solve stops on the rho-normalised residual)."""
    vel, _, _ = oracle.lattice()
    phi = np.array([oracle.basis(v) for v in vel])  # (39, 13)
    worst = 0.0
    for _ in range(300):
        u, T = random_state(RNG)
        rho = RNG.uniform(0.2, 3.0)
        m = mb_targets(u, T)
        lam, F, nu, st = oracle.newton(oracle.targets(u, T), oracle.gaussian_guess(u, T),
                                       maxit=100)
        assert st == 0
        mom = rho * (F[:, None] * phi).sum(0)
        rel = np.abs(mom - rho * m) / np.maximum(rho, np.abs(rho * m))
        worst = max(worst, rel.max())
    assert worst <= 1e-12, worst


def test_rest_state_reduces_to_1d_problem(oracle):
    """At u = 0 the solution is lam_1 = lam_3 = 0, no off-diagonal lam_2, lam_2 = b I with b
    solving sum_i e^{b|xi_i|^2}|xi_i|^2 / sum_i e^{b|xi_i|^2} = 3T (solved here by bisection),
    and lam_0 = -log sum_i e^{b|xi_i|^2}."""
    vel, _, _ = oracle.lattice()
    c2 = (vel.astype(float) ** 2).sum(1)
    for T in (0.34, 0.4, 0.5, 0.7, 1.0):
        lo, hi = -20.0, 5.0
        for _ in range(200):
            b = 0.5 * (lo + hi)
            e = np.exp(b * c2)
            if (e * c2).sum() / e.sum() > 3 * T:
                hi = b
            else:
                lo = b
        b = 0.5 * (lo + hi)
        lam0 = -np.log(np.exp(b * c2).sum())
        u = np.zeros(3)
        lam, F, nu, st = oracle.newton(oracle.targets(u, T), oracle.gaussian_guess(u, T),
                                       maxit=100)
        assert st == 0
        want = np.array([lam0, 0, 0, 0, b, b, b, 0, 0, 0, 0, 0, 0])
        assert np.allclose(lam, want, rtol=1e-11, atol=1e-11), (T, lam, want)


def test_jacobian_matches_finite_differences(oracle):
    for _ in range(10):
        u, T = random_state(RNG)
        m = oracle.targets(u, T)
        lam, F, nu, st = oracle.newton(m, oracle.gaussian_guess(u, T), maxit=100)
        lam = lam + RNG.normal(0, 1e-2, 13)
        J = oracle.jacobian(lam)
        h = 1e-6
        Jfd = np.zeros((13, 13))
        for k in range(13):
            e = np.zeros(13)
            e[k] = h
            Jfd[:, k] = (oracle.residual(lam + e, m) - oracle.residual(lam - e, m)) / (2 * h)
        assert np.allclose(J, Jfd, rtol=1e-7, atol=1e-8)
        assert np.allclose(J, J.T)
        assert np.all(np.linalg.eigvalsh(J) > 0)


def test_inverse_is_an_inverse(oracle):
    u, T = np.array([0.4, -0.3, 0.2]), 0.55
    lam, F, _, _ = oracle.newton(oracle.targets(u, T), oracle.gaussian_guess(u, T), maxit=100)
    J = oracle.jacobian(lam)
    Ji = oracle.invert(J)
    assert np.allclose(Ji @ J, np.eye(13), atol=1e-9)
    assert np.allclose(Ji, np.linalg.inv(J), rtol=1e-8, atol=1e-8)


def test_newton_converges_quadratically(oracle):
    for _ in range(5):
        u, T = random_state(RNG)
        m = oracle.targets(u, T)
        lam_ex, _, _, _ = oracle.newton(m, oracle.gaussian_guess(u, T), maxit=100)
        start = lam_ex + RNG.normal(0, 3e-4, 13)
        rs = []
        for k in range(0, 6):
            lam, F, nu, st = oracle.newton(m, start, tol=0.0, maxit=k, min_upd=k)
            rs.append(np.abs(oracle.residual(lam, m)).max())
        # r_{k+1} <= C r_k^2 while above round-off
        for a, b in zip(rs, rs[1:]):
            if a > 1e-7:
                assert b <= 50.0 * a * a, rs
        assert rs[5] < 1e-13, rs


def test_solver_equivariance_under_lattice_symmetries(oracle):
    """Mirroring x and swapping x<->y map the solution's multipliers accordingly."""
    u, T = np.array([0.5, -0.3, 0.2]), 0.6
    lam, _, _, _ = oracle.newton(oracle.targets(u, T), oracle.gaussian_guess(u, T), maxit=100)
    # mirror x: odd-in-x multipliers change sign
    um = u * np.array([-1, 1, 1])
    lm, _, _, _ = oracle.newton(oracle.targets(um, T), oracle.gaussian_guess(um, T), maxit=100)
    sign = np.array([1, -1, 1, 1, 1, 1, 1, -1, -1, 1, -1, 1, 1])
    assert np.allclose(lm, sign * lam, atol=1e-12)
    # swap x <-> y
    us = u[[1, 0, 2]]
    ls, _, _, _ = oracle.newton(oracle.targets(us, T), oracle.gaussian_guess(us, T), maxit=100)
    perm = [0, 2, 1, 3, 5, 4, 6, 7, 9, 8, 11, 10, 12]
    assert np.allclose(ls, lam[perm], atol=1e-12)


def test_equilibrium_energy_closure(oracle):
    """sum_i (f_i^eq |xi_i|^2 + g_i^eq) = rho u^2 + 2 C_v rho T (E = u^2/2 + C_v T)."""
    vel, _, _ = oracle.lattice()
    c2 = (vel.astype(float) ** 2).sum(1)
    for gamma in (1.4, 5.0 / 3.0, 1.3):
        cfg = oracle.Config(nx=1, gamma=gamma)
        cv = 1.0 / (gamma - 1.0)
        for _ in range(10):
            u, T = random_state(RNG)
            rho = RNG.uniform(0.5, 2.0)
            feq, geq, lam, st = oracle.equilibrium(cfg, rho, u, T)
            assert st == 0
            lhs = (feq * c2).sum() + geq.sum()
            rhs = rho * (u @ u) + 2 * cv * rho * T
            assert abs(lhs - rhs) <= 1e-12 * abs(rhs)
            assert np.allclose(geq, (2 * cv - 3) * T * feq, rtol=1e-15)


def test_gaussian_guess_is_normalised_maxwellian(oracle):
    vel, _, _ = oracle.lattice()
    u, T = np.array([0.2, 0.1, -0.4]), 0.5
    lam = oracle.gaussian_guess(u, T)
    F = oracle.feq_norm(lam)
    assert abs(F.sum() - 1) < 1e-14
    d2 = ((vel - u) ** 2).sum(1)
    ref = np.exp(-d2 / (2 * T))
    assert np.allclose(F, ref / ref.sum(), rtol=1e-13)
