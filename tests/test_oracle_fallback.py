"""Pins of the oracle's fallback equilibrium: where the 13-moment equilibrium does not exist
(outside the moment cone of the 39 velocities), a cell relaxes to the maximum-entropy
equilibrium under the five collision invariants [1, xi, |xi|^2] (a reading; the paper does not
say what a cell does when its constraint solve fails)."""
import numpy as np
from scipy.optimize import linprog

RNG = np.random.default_rng(17)
# states found outside the cone: behind a NACA0012 at Ma 1.5 (T_inf = 0.5) and in the
# rms-Ma-0.8 box
OUTSIDE = [((1.416, -0.348, 0.0), 0.414), ((-0.401, 0.936, -0.488), 0.397)]


def _invariants(vel, F):
    v = vel.astype(float)
    return np.array([F.sum(), F @ v[:, 0], F @ v[:, 1], F @ v[:, 2], F @ (v ** 2).sum(1)])


def _in_cone(oracle, u, T):
    """True if some strictly positive weights on the 39 velocities have the 13 target moments
    (linear programme: maximise the smallest weight)."""
    vel, _, _ = oracle.lattice()
    Phi = np.array([oracle.basis(v) for v in np.asarray(vel, np.int32)])
    m = oracle.targets(np.asarray(u, float), T)
    A_eq = np.hstack([Phi.T, np.zeros((13, 1))])
    A_ub = np.hstack([-np.eye(39), np.ones((39, 1))])
    res = linprog(np.r_[np.zeros(39), -1.0], A_ub=A_ub, b_ub=np.zeros(39), A_eq=A_eq, b_eq=m,
                  bounds=[(0, None)] * 39 + [(None, None)], method="highs")
    return res.status == 0 and -res.fun > 1e-12


def test_outside_states_are_outside_the_cone_and_fail_the_full_solve(oracle):
    for u, T in OUTSIDE:
        assert not _in_cone(oracle, u, T)
        m = oracle.targets(np.asarray(u), T)
        assert oracle.newton(m, oracle.gaussian_guess(np.asarray(u), T), maxit=1000)[3] == 1
    assert _in_cone(oracle, (1.0, 0.2, 0.0), 0.5)


def test_fallback_reproduces_the_five_invariants(oracle):
    vel, _, _ = oracle.lattice()
    states = list(OUTSIDE) + [(tuple(RNG.uniform(-1.2, 1.2, 3)), RNG.uniform(0.3, 1.0))
                              for _ in range(200)]
    for u, T in states:
        u = np.asarray(u)
        mu, F, n, st = oracle.newton5(u, T)
        assert st == 0
        want = np.r_[1.0, u, u @ u + 3 * T]
        assert np.all(np.abs(_invariants(vel, F) - want) <= 1e-12 * np.maximum(1, np.abs(want)))


def test_fallback_equals_full_equilibrium_at_rest(oracle):
    """At u = 0 the isotropic exp(mu_0 + b|xi|^2) satisfies all 13 constraints (cubic symmetry
    of the velocity set), so by uniqueness it is the 13-moment equilibrium."""
    for T in (0.36, 0.5, 0.8, 1.1):
        u = np.zeros(3)
        F5 = oracle.newton5(u, T)[1]
        lam, F13, n, st = oracle.newton(oracle.targets(u, T), oracle.gaussian_guess(u, T),
                                        maxit=200)
        assert st == 0
        assert np.allclose(F5, F13, rtol=1e-12, atol=0)


def test_collision_outside_the_cone_conserves(oracle):
    """A failed 13-moment solve is still reported, and the collision conserves mass, momentum
    and energy to round-off through the fallback."""
    vel, _, _ = oracle.lattice()
    cfg = oracle.Config(nx=1, tau=0.6, kn_sensor=1)
    cv = 1.0 / (cfg.gamma - 1.0)
    for (u, T), rho in zip(OUTSIDE, (0.954, 0.6)):
        u = np.asarray(u)
        F = oracle.newton5(u, T)[1]
        f = rho * F * (1 + 1e-3 * RNG.uniform(-1, 1, 39))
        g = (2 * cv - 3) * T * rho * F
        lam = oracle.gaussian_guess(u, T)
        fs, gs, lam2, nu, eps, al, st, fb = oracle.collide_cell(cfg, f, g, lam)
        assert st == 1 and fb
        c2 = (vel.astype(float) ** 2).sum(1)
        m0 = np.r_[_invariants(vel, f)[:4], f @ c2 + g.sum()]
        m1 = np.r_[_invariants(vel, fs)[:4], fs @ c2 + gs.sum()]
        assert np.all(np.abs(m1 - m0) <= 1e-13 * np.maximum(1, np.abs(m0))), m1 - m0


def test_failed_cell_keeps_embedded_fallback_multipliers_and_retries_cheaply(oracle):
    """After a fallback the 13 multipliers are the five embedded (lambda_4..6 equal, the rest of
    the second and third orders zero), so exp(Phi lambda) is the fallback equilibrium, and the cell
    is flagged; the next collision of a cell still outside the cone spends at most the Newton
    budget on a retry step and no update off one."""
    vel, _, _ = oracle.lattice()
    cfg = oracle.Config(nx=1, tau=0.6, kn_sensor=1)
    cv = 1.0 / (cfg.gamma - 1.0)
    (u, T), rho = OUTSIDE[0], 0.954
    u = np.asarray(u)
    F5 = oracle.newton5(u, T)[1]
    f, g = rho * F5, (2 * cv - 3) * T * rho * F5
    lam = oracle.gaussian_guess(u, T)
    lam[7] = 1e-3  # an unflagged cell: the full budget
    fs, gs, lam2, nu, eps, al, st, fb = oracle.collide_cell(cfg, f, g, lam)
    assert st == 1 and fb and nu > 3
    assert np.all(lam2[7:] == 0) and lam2[4] == lam2[5] == lam2[6]
    F = oracle.feq_norm(lam2)
    want = np.r_[1.0, u, u @ u + 3 * T]
    assert np.all(np.abs(_invariants(vel, F) - want) <= 1e-12 * np.maximum(1, np.abs(want)))
    for t, most in ((0, cfg.newton_maxit), (5, 0)):
        _, _, lam3, nu2, _, _, st2, fb2 = oracle.collide_cell(cfg, f, g, lam2, on_fallback=True,
                                                              t=t)
        assert st2 == 1 and fb2 and nu2 <= most
        assert np.all(lam3[7:] == 0) and np.allclose(oracle.feq_norm(lam3), F, rtol=1e-12, atol=0)


def test_a_solved_rest_state_is_not_taken_for_a_fallback(oracle):
    """A cell at rest has multipliers of the embedded shape; unflagged, it keeps the full Newton
    budget when a strong change arrives (the flag, not the shape, identifies a fallback)."""
    cfg = oracle.Config(nx=1, tau=0.6, kn_sensor=1)
    feq, geq, lam, st = oracle.equilibrium(cfg, 1.0, np.zeros(3), 0.5)
    assert st == 0
    lam[7:] = 0.0           # the exact shape that symmetric arithmetic gives at rest
    lam[5] = lam[6] = lam[4]
    # a cell at rest receives populations of a fast, hot state (a shock arriving)
    f2, g2, _, _ = oracle.equilibrium(cfg, 2.5, np.array([0.9, 0.0, 0.0]), 0.8)
    fs, gs, lam2, nu, eps, al, st, fb = oracle.collide_cell(cfg, f2, g2, lam, t=3)
    assert st == 0 and not fb and nu > 3


def _flagged_outside_cell(oracle):
    cfg = oracle.Config(nx=1, tau=0.6, kn_sensor=1)
    cv = 1.0 / (cfg.gamma - 1.0)
    (u, T), rho = OUTSIDE[0], 0.954
    u = np.asarray(u)
    F5 = oracle.newton5(u, T)[1]
    f, g = rho * F5, (2 * cv - 3) * T * rho * F5
    lam = oracle.gaussian_guess(u, T)
    lam2, fb = oracle.collide_cell(cfg, f, g, lam)[2::5]
    assert fb
    return cfg, f, g, lam2


def test_flagged_cell_retries_on_multiples_of_eight(oracle):
    """The failure policy's schedule: a flagged cell tries the full solve (with the Newton
    budget; outside the cone it runs out or the line search gives up) exactly on the time steps
    that are multiples of 8, and takes no update on every other step."""
    cfg, f, g, lam2 = _flagged_outside_cell(oracle)
    for t in range(0, 33):
        nu, st, fb = (lambda r: (r[3], r[6], r[7]))(
            oracle.collide_cell(cfg, f, g, lam2, on_fallback=True, t=t))
        assert st == 1 and fb
        if t % 8 == 0:
            assert 1 <= nu <= cfg.newton_maxit, (t, nu)
        else:
            assert nu == 0, (t, nu)


def test_retry_schedule_is_the_same_for_every_cell(oracle):
    """On a lattice every flagged cell follows the same schedule, wherever it sits: a periodic
    row of identical cells outside the cone keeps identical populations and multipliers after
    each step (no cell-index dependence), and its Newton updates per step are 0 off the retry
    steps."""
    cfg1, f, g, lam2 = _flagged_outside_cell(oracle)
    n = 70
    cfg = oracle.Config(nx=n, ny=1, nz=1, tau=0.6, kn_sensor=1)
    st = oracle.State(cfg, np.zeros(n, np.uint8), np.tile(f, (n, 1)), np.tile(g, (n, 1)),
                      np.tile(lam2, (n, 1)), on_fb=np.ones(n, np.uint8))
    prev = 0
    for t in range(10):
        oracle.step(st, 1)
        assert (st.f == st.f[0]).all() and (st.lam == st.lam[0]).all()
        upd = st.stats.newton_updates - prev
        prev = st.stats.newton_updates
        assert (upd == 0) == (t % 8 != 0), (t, upd)
        assert st.on_fb.all()


def test_a_flagged_cell_back_inside_the_cone_returns_at_its_retry_step(oracle):
    """A flagged cell whose state lies inside the cone (|u| ~ 1, T = 0.5) and whose stored
    multipliers are the fallback embedding of that same state: from the embedding the full solve
    needs 5-7 Newton updates, so on its next retry step (t = 16) it converges with the full
    budget, is unflagged and relaxes to the 13-moment equilibrium; off a retry step (t = 17)
    it stays on the fallback."""
    vel, _, _ = oracle.lattice()
    cfg = oracle.Config(nx=1, tau=0.6, kn_sensor=1)
    cv = 1.0 / (cfg.gamma - 1.0)
    for u, T in (((1.0, 0.3, 0.0), 0.5), ((0.8, 0.5, 0.1), 0.5), ((1.1, 0.4, 0.0), 0.42)):
        u = np.asarray(u)
        mu = oracle.newton5(u, T)[0]
        lam = np.r_[mu[:4], mu[4], mu[4], mu[4], np.zeros(6)]
        F13 = oracle.newton(oracle.targets(u, T), oracle.gaussian_guess(u, T), maxit=200)[1]
        f, g = F13, (2 * cv - 3) * T * F13  # rho = 1, at the 13-moment equilibrium
        n_full = oracle.newton(oracle.targets(u, T), lam, maxit=30)[2]
        assert n_full > 3
        _, _, lam2, nu, _, _, st, fb = oracle.collide_cell(cfg, f, g, lam, on_fallback=True, t=16)
        assert st == 0 and not fb and nu == n_full
        assert np.allclose(oracle.feq_norm(lam2), F13, rtol=1e-10, atol=0)
        _, _, lam3, nu3, _, _, st3, fb3 = oracle.collide_cell(cfg, f, g, lam, on_fallback=True,
                                                              t=17)
        assert st3 == 1 and fb3 and nu3 == 0


def test_fallback_region_does_not_stick(oracle):
    """The small Ma 2 airfoil: cells leave the moment cone behind the shock during the start-up
    and take the fallback; once the flow has settled they come back inside the cone, and the
    policy returns them to the 13-moment equilibrium (no cell flagged at step 200, none failing
    after step 100).  With a retry budget of 3 updates the same run kept 768 cells (17% of the
    lattice) on the fallback at every step, every one of them strictly inside the cone."""
    from paper_1910_13515_gb300 import inputs
    s = inputs.naca(nx=96, ny=48, chord=24, x_le=24, mach=2.0)
    cfg = oracle.Config(nx=s.nx, ny=s.ny, nz=s.nz, periodic=s.periodic, gamma=s.gamma, tau=s.tau,
                        kn_sensor=s.kn_sensor, rho_inf=s.rho_inf, u_inf=s.u_inf, T_inf=s.T_inf)
    st = oracle.init(cfg, s.mask, s.rho, s.u, s.T)
    assert oracle.step(st, 50) > 0  # the start-up leaves the cone
    oracle.step(st, 50)
    assert oracle.step(st, 100) == 0
    assert st.on_fb.sum() == 0
