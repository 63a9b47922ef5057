"""Pins of the oracle's fourth-order polynomial-equilibrium DDF-BGK model (the paper's
comparison model, Sec. 5) against mathematics independent of the oracle: Maxwell-Boltzmann
moments by Gauss-Hermite quadrature, the Hermite projection integral, the weights' rest
state, conservation, and the sound speed and viscosity the model must produce."""
import itertools
import math

import numpy as np
import pytest
from numpy.polynomial.hermite import hermgauss

RNG = np.random.default_rng(2027)


@pytest.fixture(scope="module")
def poly():
    from oracle import oracle39, poly39
    oracle39.build()
    return poly39


def gauss_nodes(mean, var, n=8):
    """Tensor Gauss-Hermite nodes (n^3, 3) and weights (n^3,) of the normal density
    N(mean, var I): exact for polynomials of degree <= 2n - 1 per axis."""
    x, w = hermgauss(n)
    s = math.sqrt(2.0 * var)
    pts = np.array(list(itertools.product(range(n), repeat=3)))
    xi = np.asarray(mean)[None, :] + s * x[pts]
    W = np.prod(w[pts], axis=1) / math.pi**1.5
    return xi, W


def monomials(max_degree):
    return [k for k in itertools.product(range(max_degree + 1), repeat=3) if sum(k) <= max_degree]


def mono(xi, k):
    return xi[:, 0] ** k[0] * xi[:, 1] ** k[1] * xi[:, 2] ** k[2]


def mb_moment(rho, u, T, k):
    """int xi^k f^MB d^3xi of rho N(u, T I), by quadrature."""
    xi, W = gauss_nodes(u, T)
    return rho * float((mono(xi, k) * W).sum())


def random_states(n, umax=0.6, T=(0.45, 0.9)):
    rho = RNG.uniform(0.5, 2.0, n)
    u = RNG.uniform(-umax, umax, (n, 3))
    Ts = RNG.uniform(*T, n)
    return rho, u, Ts


def test_reference_temperature_is_the_weights_second_moment(poly):
    vel, w = poly.lattice()
    assert abs((w * vel[:, 0] ** 2).sum() - poly.THETA0) < 1e-15
    assert abs(w.sum() - 1.0) < 1e-15


def test_lattice_moments_to_third_order_are_maxwellian(poly):
    """The D3Q39 quadrature is exact to degree 7, so every moment of order <= 3 of the
    fourth-order equilibrium equals the Maxwellian's (all 20 of them, for any u and T)."""
    vel, _ = poly.lattice()
    rho, u, T = random_states(40)
    f = poly.feq(rho, u, T)
    for n in range(40):
        for k in monomials(3):
            got = float((f[n] * mono(vel, k)).sum())
            want = mb_moment(rho[n], u[n], T[n], k)
            assert abs(got - want) <= 1e-13 * max(1.0, abs(want)) * rho[n], (n, k, got, want)


def test_continuous_expansion_has_the_maxwellian_moments_to_fourth_order(poly):
    """Over the continuum, Gaussian weight N(0, theta0) times the truncated expansion has
    the Maxwellian's moments up to the truncation order: this pins a^(4), H^(4) and the
    1/(n! theta0^n) normalisation, which the lattice moments of order <= 3 cannot see."""
    xi, W = gauss_nodes(np.zeros(3), poly.THETA0, n=8)
    rho, u, T = random_states(12, umax=0.8, T=(0.3, 1.2))
    P = poly.expansion(xi, rho, u, T)
    for n in range(len(rho)):
        for k in monomials(4):
            got = float((P[n] * mono(xi, k) * W).sum())
            want = mb_moment(rho[n], u[n], T[n], k)
            assert abs(got - want) <= 1e-12 * max(1.0, abs(want)) * rho[n], (n, k, got, want)
        # and not beyond: a fifth-order moment of the truncated series differs
    k5 = (5, 0, 0)
    got = float((P[0] * mono(xi, k5) * W).sum())
    assert abs(got - mb_moment(rho[0], u[0], T[0], k5)) > 1e-6


def test_coefficients_are_the_hermite_projection_of_the_maxwellian(poly):
    """a^(n) = int f^MB H^(n) dxi, the integral taken by quadrature over N(u, T I)."""
    rho, u, T = random_states(5, umax=0.8, T=(0.3, 1.2))
    a = poly.mb_coefficients(rho, u, T)
    for n in range(len(rho)):
        xi, W = gauss_nodes(u[n], T[n])
        H = poly.hermite(xi)
        for order in range(5):
            want = rho[n] * np.tensordot(W, H[order], axes=(0, 0))
            np.testing.assert_allclose(a[order][n], want, rtol=0, atol=1e-12 * rho[n])


def test_rest_state_at_the_reference_temperature_is_rho_times_the_weights(poly):
    _, w = poly.lattice()
    f = poly.feq(np.array([1.7]), np.zeros((1, 3)), np.array([poly.THETA0]))
    np.testing.assert_allclose(f[0], 1.7 * w, rtol=2e-15, atol=0)


def test_equilibrium_energy_and_mirror_equivariance(poly):
    vel, _ = poly.lattice()
    cfg = poly.Config(nx=1, gamma=1.4)
    rho, u, T = random_states(20)
    f, g = poly.equilibrium(cfg, rho, u.T, T)
    e2 = f @ (vel**2).sum(axis=1) + g.sum(axis=1)
    cv = 1.0 / (cfg.gamma - 1.0)
    np.testing.assert_allclose(e2, rho * (u**2).sum(axis=1) + 2 * cv * rho * T, rtol=1e-13)
    # x -> -x maps velocity i to the one with the x component negated
    mirror = [int(np.where((vel == vel[i] * np.array([-1, 1, 1])).all(axis=1))[0][0])
              for i in range(len(vel))]
    um = u * np.array([-1.0, 1.0, 1.0])
    fm, _ = poly.equilibrium(cfg, rho, um.T, T)
    np.testing.assert_allclose(fm, f[:, mirror], rtol=1e-14, atol=1e-16)


def test_collision_conserves_mass_momentum_energy(poly):
    vel, _ = poly.lattice()
    cfg = poly.Config(nx=1, gamma=1.4, tau=0.57)
    rho, u, T = random_states(30, umax=0.4, T=(0.55, 0.8))
    f, g = poly.equilibrium(cfg, rho, u.T, T)
    f = f * (1 + 0.05 * RNG.uniform(-1, 1, f.shape))
    g = g * (1 + 0.05 * RNG.uniform(-1, 1, g.shape))
    fs, gs = poly.collide(cfg, f, g)
    for a, b in ((f, fs),):
        np.testing.assert_allclose(b.sum(axis=1), a.sum(axis=1), rtol=1e-14)
        np.testing.assert_allclose(b @ vel, a @ vel, rtol=0, atol=1e-14)
    e = f @ (vel**2).sum(axis=1) + g.sum(axis=1)
    es = fs @ (vel**2).sum(axis=1) + gs.sum(axis=1)
    np.testing.assert_allclose(es, e, rtol=1e-14)


def test_uniform_flow_is_invariant(poly):
    cfg = poly.Config(nx=5, ny=4, nz=3, tau=0.6)
    N = cfg.ncells
    u = np.tile(np.array([[0.3], [-0.2], [0.1]]), (1, N))
    st = poly.init(cfg, np.full(N, 1.1), u, np.full(N, 0.6))
    f0 = st.f.copy()
    poly.step(st, 20)
    np.testing.assert_allclose(st.f, f0, rtol=1e-13, atol=0)
    rho, uu, T = poly.macros(cfg, st.f, st.g)
    np.testing.assert_allclose(uu, u, atol=1e-14)
    np.testing.assert_allclose(T, 0.6, rtol=1e-13)


def test_streaming_moves_each_population_by_its_velocity(poly):
    """Brute force on a tiny periodic lattice: tagged values land at x + xi_i (mod n)."""
    vel, _ = poly.lattice()
    cfg = poly.Config(nx=5, ny=4, nz=3)
    N = cfg.ncells
    h = np.arange(N * 39, dtype=np.float64).reshape(N, 39)
    out = poly.stream(cfg, h)
    for c in range(N):
        x, y, z = c % 5, (c // 5) % 4, c // 20
        for i in range(39):
            cx, cy, cz = (int(v) for v in vel[i])
            d = (x + cx) % 5 + 5 * ((y + cy) % 4) + 20 * ((z + cz) % 3)
            assert out[d, i] == h[c, i]


def test_sound_speed(poly):
    """A standing acoustic wave oscillates with c_s = sqrt(gamma T)."""
    L, gamma = 48, 1.4
    T0 = poly.THETA0
    cfg = poly.Config(nx=L, gamma=gamma, tau=0.52)
    x = np.arange(L)
    k = 2 * np.pi / L
    rho = 1 + 1e-4 * np.cos(k * x)
    st = poly.init(cfg, rho, np.zeros((3, L)), T0 * rho ** (gamma - 1))
    amps = []
    for _ in range(70):
        r, _, _ = poly.macros(cfg, st.f, st.g)
        amps.append(((r - 1) * np.cos(k * x)).sum())
        poly.step(st, 1)
    amps = np.array(amps)
    i = np.where((amps[:-1] > 0) & (amps[1:] <= 0))[0][0]
    tq = i + amps[i] / (amps[i] - amps[i + 1])
    c = (L / 4) / tq
    assert abs(c / math.sqrt(gamma * T0) - 1) < 0.02, (c, math.sqrt(gamma * T0))


@pytest.mark.parametrize("T0", [2.0 / 3.0, 0.55])
def test_shear_wave_viscosity(poly, T0):
    """A transverse shear wave decays at exp(-nu k^2 t) with nu = (tau - 1/2) T: the third
    moments of this equilibrium are the Maxwellian's, so the BGK viscosity is exact."""
    L, tau = 32, 0.8
    cfg = poly.Config(nx=L, tau=tau)
    x = np.arange(L)
    k = 2 * np.pi / L
    u = np.zeros((3, L))
    u[1] = 1e-3 * np.sin(k * x)
    st = poly.init(cfg, np.ones(L), u, np.full(L, T0))
    amp = {}
    for t in (10, 110):
        poly.step(st, t - st.t)
        _, uu, _ = poly.macros(cfg, st.f, st.g)
        amp[t] = (uu[1] * np.sin(k * x)).sum()
    nu = -math.log(amp[110] / amp[10]) / (k * k * 100)
    assert abs(nu / ((tau - 0.5) * T0) - 1) < 0.02, (nu, (tau - 0.5) * T0)
