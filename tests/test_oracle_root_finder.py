"""Pins of the oracle's other root finders (lbm39 root_finder 1-3; the paper's outlook
names other root finders): it must land on the same constrained maximum-entropy equilibrium as
Newton-Raphson -- the one the closed-form Maxwell-Boltzmann targets define, unique because the
dual problem is strictly convex -- under the same stopping rule, forming fewer Jacobians."""
import numpy as np

from paper_1910_13515_gb300 import inputs

RNG = np.random.default_rng(314)


def mb_targets(u, T):
    """13 Maxwell-Boltzmann moments per unit density, written out (Eq. 13constraints with the
    contracted third moment u (u^2 + 5 T))."""
    u = np.asarray(u, float)
    uu = np.outer(u, u) + T * np.eye(3)
    return np.r_[1.0, u, uu[0, 0], uu[1, 1], uu[2, 2], uu[0, 1], uu[0, 2], uu[1, 2],
                 u * (u @ u + 5 * T)]


def moments(vel, F):
    v = vel.astype(float)
    phi = np.stack([np.ones(39), v[:, 0], v[:, 1], v[:, 2], v[:, 0] ** 2, v[:, 1] ** 2,
                    v[:, 2] ** 2, v[:, 0] * v[:, 1], v[:, 0] * v[:, 2], v[:, 1] * v[:, 2],
                    *(v.T * (v ** 2).sum(1))])
    return phi @ F


def random_state(rng):
    T = rng.uniform(0.4, 0.9)
    u = rng.normal(size=3)
    u *= rng.uniform(0, 1.0) / max(np.linalg.norm(u), 1e-12)
    return u, T


def test_hybrid_reaches_the_maxwell_boltzmann_moments(oracle):
    vel, _, _ = oracle.lattice()
    for _ in range(300):
        u, T = random_state(RNG)
        m = mb_targets(u, T)
        lam, F, n, nj, st = oracle.newton_hybrid(m, oracle.gaussian_guess(u, T), maxit=200)
        assert st == 0
        assert np.all(np.abs(moments(vel, F) - m) <= 1e-12 * np.maximum(1, np.abs(m)))


def test_hybrid_and_newton_find_the_same_equilibrium_from_warm_starts(oracle):
    """From the multipliers of a nearby state (a warm start, as between time steps) both root
    finders converge; the equilibria agree to 1e-12 and the hybrid forms fewer Jacobians."""
    n_upd = n_jac = n_newton = 0
    for _ in range(300):
        u, T = random_state(RNG)
        lam0 = oracle.newton(mb_targets(u, T), oracle.gaussian_guess(u, T), maxit=200)[0]
        du = RNG.normal(scale=0.02, size=3)
        dT = RNG.normal(scale=0.01)
        m = mb_targets(u + du, T + dT)
        l1, F1, k1, s1 = oracle.newton(m, lam0)
        l2, F2, k2, j2, s2 = oracle.newton_hybrid(m, lam0)
        assert s1 == 0 and s2 == 0
        assert np.abs(F1 - F2).max() <= 1e-12 * F1.max()
        n_upd += k2
        n_jac += j2
        n_newton += k1
    assert n_jac <= 0.8 * n_newton, (n_jac, n_newton)  # fewer Jacobians than Newton forms


def test_hybrid_at_rest_is_the_isotropic_solution(oracle):
    """u = 0: lambda_1 = lambda_3 = 0 and lambda_2 = b I with sum e^{b|xi|^2}|xi|^2 / sum
    e^{b|xi|^2} = 3 T (bisection), from a warm start at another temperature."""
    vel, _, _ = oracle.lattice()
    c2 = (vel.astype(float) ** 2).sum(1)
    for T in (0.4, 0.55, 0.8):
        lo, hi = -20.0, 0.0
        for _ in range(200):
            b = 0.5 * (lo + hi)
            w = np.exp(b * (c2 - c2.max()))
            if (w * c2).sum() / w.sum() > 3 * T:
                hi = b
            else:
                lo = b
        lam0 = oracle.newton(mb_targets(np.zeros(3), 1.05 * T),
                             oracle.gaussian_guess(np.zeros(3), 1.05 * T), maxit=200)[0]
        lam, F, n, nj, st = oracle.newton_hybrid(mb_targets(np.zeros(3), T), lam0)
        assert st == 0
        assert np.abs(lam[[1, 2, 3, 7, 8, 9, 10, 11, 12]]).max() < 1e-12
        assert np.allclose(lam[4:7], 0.5 * (lo + hi), rtol=1e-10, atol=0)


def test_lattice_run_with_the_hybrid_matches_newton(oracle):
    """A periodic box stepped 20 times with either root finder: the same flow to 1e-12 (both
    converge each solve below the 1e-12 residual, polished)."""
    s = inputs.box(seed=0, shape=(10, 10, 10))
    runs = []
    for rf in (0, 1):
        cfg = oracle.Config(nx=s.nx, ny=s.ny, nz=s.nz, gamma=s.gamma, tau=s.tau,
                            kn_sensor=s.kn_sensor, root_finder=rf)
        st = oracle.init(cfg, s.mask, s.rho, s.u, s.T)
        assert oracle.step(st, 20) == 0
        runs.append((oracle.macros(st), st.stats.newton_updates))
    (a, na), (b, nb) = runs
    for x, y in zip(a[:3], b[:3]):
        assert np.abs(x - y).max() <= 1e-12 * max(np.abs(y).max(), 1.0)
    assert nb >= na  # the hybrid takes more (cheaper) updates


def test_fp32_direction_reaches_the_same_equilibrium(oracle):
    """Newton with a single-precision direction (root_finder 2): the residual that decides
    convergence is the double-precision one, so it lands on the Maxwell-Boltzmann moments to
    1e-12 and on Newton's equilibrium, from cold and warm starts."""
    vel, _, _ = oracle.lattice()
    extra = 0
    for _ in range(200):
        u, T = random_state(RNG)
        m = mb_targets(u, T)
        lam, F, n, st = oracle.newton_fp32dir(m, oracle.gaussian_guess(u, T), maxit=200)
        assert st == 0
        assert np.all(np.abs(moments(vel, F) - m) <= 1e-12 * np.maximum(1, np.abs(m)))
        lam0 = lam
        m2 = mb_targets(u + RNG.normal(scale=0.02, size=3), T + RNG.normal(scale=0.01))
        l1, F1, k1, s1 = oracle.newton(m2, lam0)
        l2, F2, k2, s2 = oracle.newton_fp32dir(m2, lam0)
        assert s1 == 0 and s2 == 0
        assert np.abs(F1 - F2).max() <= 1e-12 * F1.max()
        extra += k2 - k1
    assert extra >= 0  # a linear rate: never fewer updates than Newton in total


def test_lattice_run_with_the_fp32_direction_matches_newton(oracle):
    s = inputs.box(seed=3, shape=(10, 10, 10))
    runs = []
    for rf in (0, 2):
        cfg = oracle.Config(nx=s.nx, ny=s.ny, nz=s.nz, gamma=s.gamma, tau=s.tau,
                            kn_sensor=s.kn_sensor, root_finder=rf)
        st = oracle.init(cfg, s.mask, s.rho, s.u, s.T)
        assert oracle.step(st, 20) == 0
        runs.append(oracle.macros(st))
    for x, y in zip(runs[0][:3], runs[1][:3]):
        assert np.abs(x - y).max() <= 1e-12 * max(np.abs(y).max(), 1.0)


def test_fp32_start_reaches_the_same_equilibrium(oracle):
    """Newton after a single-precision start (root_finder 3): the float steps only move the
    starting point, and the double-precision residual decides convergence, so it lands on the
    Maxwell-Boltzmann moments to 1e-12 and on Newton's equilibrium from cold and warm starts."""
    vel, _, _ = oracle.lattice()
    for _ in range(200):
        u, T = random_state(RNG)
        m = mb_targets(u, T)
        lam, F, n, n32, st = oracle.newton_fp32start(m, oracle.gaussian_guess(u, T), maxit=200)
        assert st == 0
        assert np.all(np.abs(moments(vel, F) - m) <= 1e-12 * np.maximum(1, np.abs(m)))
        m2 = mb_targets(u + RNG.normal(scale=0.05, size=3), T + RNG.normal(scale=0.02))
        l1, F1, k1, s1 = oracle.newton(m2, lam)
        l3, F3, k3, n3, s3 = oracle.newton_fp32start(m2, lam)
        assert s1 == 0 and s3 == 0
        assert np.abs(F1 - F3).max() <= 1e-12 * F1.max()


def test_fp32_start_saves_double_precision_updates(oracle):
    """Warm starts a time step away in a fast flow (residuals ~1e-2): the float steps take the
    residual to about 1e-4, and the double-precision updates that remain are at least a
    quarter fewer than those of the same solver without the float start (root_finder 2).
    (A residual near 1, where an undamped step overshoots, may take none: the damped
    double-precision iteration then starts from the warm start itself.)"""
    n2 = n3 = n32 = 0
    for _ in range(200):
        u, T = random_state(RNG)
        lam0 = oracle.newton(mb_targets(u, T), oracle.gaussian_guess(u, T), maxit=200)[0]
        m = mb_targets(u + RNG.normal(scale=0.1, size=3), T + RNG.normal(scale=0.03))
        r0 = np.abs(oracle.residual(lam0, m)).max()
        l2, F2, k2, s2 = oracle.newton_fp32dir(m, lam0)
        l3, F3, k3, j3, s3 = oracle.newton_fp32start(m, lam0)
        assert s2 == 0 and s3 == 0
        assert np.abs(F2 - F3).max() <= 1e-12 * F2.max()
        if 1e-4 <= r0 < 0.1:
            assert j3 >= 1  # above the threshold, within reach of a full step: a float step
        n2 += k2
        n3 += k3
        n32 += j3
    assert n3 <= 0.75 * n2, (n3, n2)
    assert n32 >= 200


def test_fp32_start_leaves_converged_and_unbudgeted_solves_alone(oracle):
    """A warm start already at the root takes no float step and no update; a solve with no
    budget (a cell on the fallback off a retry step) takes no float step and keeps lambda."""
    for _ in range(50):
        u, T = random_state(RNG)
        m = mb_targets(u, T)
        lam = oracle.newton(m, oracle.gaussian_guess(u, T), maxit=200)[0]
        l3, F3, k3, j3, s3 = oracle.newton_fp32start(m, lam)
        assert (k3, j3, s3) == (0, 0, 0) and np.array_equal(l3, lam)
        m2 = mb_targets(u + 0.1, T)
        l4, F4, k4, j4, s4 = oracle.newton_fp32start(m2, lam, maxit=0)
        assert (k4, j4, s4) == (0, 0, 1) and np.array_equal(l4, lam)


def test_lattice_run_with_the_fp32_start_matches_newton(oracle):
    s = inputs.box(seed=5, shape=(10, 10, 10))
    runs = []
    for rf in (0, 3):
        cfg = oracle.Config(nx=s.nx, ny=s.ny, nz=s.nz, gamma=s.gamma, tau=s.tau,
                            kn_sensor=s.kn_sensor, root_finder=rf)
        st = oracle.init(cfg, s.mask, s.rho, s.u, s.T)
        assert oracle.step(st, 20) == 0
        runs.append((oracle.macros(st), st.stats.newton_updates))
    (a, na), (b, nb) = runs
    for x, y in zip(a[:3], b[:3]):
        assert np.abs(x - y).max() <= 1e-12 * max(np.abs(y).max(), 1.0)
    assert nb < na  # fewer double-precision updates than Newton's
