"""Parity of the CUDA polynomial-equilibrium comparison model (lbm39_poly.h) with its FP64 CPU
oracle (oracle/poly39.py), through the C ABI.

Tolerance: max relative difference <= 1e-11 in rho, u, T (u relative to max(|u|, c_s)), the
bound of the 13-moment FP64 path; the two sides differ only in the order of rounding."""
import numpy as np
import pytest

from gpu_helpers import TOL, rel_diffs
from paper_1910_13515_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def PL():
    from paper_1910_13515_gb300 import build
    build.build()
    from paper_1910_13515_gb300.lattice import PolyLattice
    return PolyLattice


@pytest.fixture(scope="module")
def poly():
    from oracle import oracle39, poly39
    oracle39.build()
    return poly39


def run_both(PL, poly, s, nsteps):
    L = PL(s.nx, s.ny, s.nz, gamma=s.gamma, tau=s.tau)
    L.init(s.rho, s.u, s.T)
    L.step(nsteps)
    g = L.read_numpy()
    cfg = poly.Config(nx=s.nx, ny=s.ny, nz=s.nz, gamma=s.gamma, tau=s.tau)
    st = poly.init(cfg, s.rho, s.u, s.T)
    poly.step(st, nsteps)
    return L, g, st, poly.macros(cfg, st.f, st.g)


@pytest.mark.parametrize("shape,seed", [((44, 26, 1), 0), ((11, 10, 9), 1)])
def test_poly_parity_100_steps(PL, poly, shape, seed):
    s = inputs.subsonic_box(*shape, seed=seed)
    _, g, _, o = run_both(PL, poly, s, 100)
    d = rel_diffs(g, o, np.zeros(s.ncells, np.uint8), s.gamma)
    assert max(d) <= TOL, d


@pytest.mark.parametrize("nsteps", [0, 1, 2, 3, 7])
def test_poly_parity_at_both_aa_parities(PL, poly, nsteps):
    s = inputs.subsonic_box(5, 6, 7, seed=4, mach_rms=0.5)
    _, g, _, o = run_both(PL, poly, s, nsteps)
    d = rel_diffs(g, o, np.zeros(s.ncells, np.uint8), s.gamma)
    assert max(d) <= TOL, d


def test_poly_conserved_sums_match_oracle_and_are_kept(PL, poly):
    s = inputs.subsonic_box(40, 30, 2, seed=2)
    L, _, st, _ = run_both(PL, poly, s, 0)
    c0 = L.conserved()
    o0 = poly.conserved(st)
    np.testing.assert_allclose(c0, o0, rtol=1e-13, atol=1e-11)
    L.step(101)
    c1 = L.conserved()
    assert L.time == 101
    assert abs(c1[0] - c0[0]) <= 1e-13 * abs(c0[0])
    assert abs(c1[4] - c0[4]) <= 1e-13 * abs(c0[4])
    assert np.abs(c1[1:4] - c0[1:4]).max() <= 1e-12 * c0[0]


def test_poly_uniform_flow_is_invariant(PL):
    L = PL(8, 6, 4, tau=0.55)
    N = 8 * 6 * 4
    u = np.tile(np.array([[0.35], [-0.25], [0.1]]), (1, N))
    L.init(np.full(N, 1.2), u, np.full(N, 0.6))
    L.step(500)
    rho, uu, T, p = L.read_numpy()
    assert np.abs(rho - 1.2).max() < 1e-13 and np.abs(T - 0.6).max() < 1e-13
    assert np.abs(uu - u).max() < 1e-13
    np.testing.assert_allclose(p, rho * T, rtol=1e-15)


def test_poly_full_size_sampled_cells_match_oracle(PL, poly):
    """At the benchmark size (2048 x 2048 x 1, the launch configuration bench.py times): after
    3 steps, sampled cells against the oracle run on the 19 x 19 periodic patch around each
    (the 3-step dependence cone has radius 9, so the patch's wrap never reaches the centre)."""
    nx = ny = 2048
    s = inputs.subsonic_box(nx, ny, 1, seed=0)
    L = PL(nx, ny, 1, gamma=s.gamma, tau=s.tau)
    L.init(s.rho, s.u, s.T)
    L.step(3)
    rho, u, T, _ = L.read_numpy()
    rng = np.random.default_rng(7)
    cells = np.concatenate([[0, nx - 1, nx * ny - 1, nx * (ny - 1)],
                            rng.integers(0, nx * ny, 28)])
    cfg = poly.Config(nx=19, ny=19, nz=1, gamma=s.gamma, tau=s.tau)
    off = np.arange(-9, 10)
    for c in cells:
        x, y = int(c % nx), int(c // nx)
        idx = (((y + off)[:, None] % ny) * nx + ((x + off)[None, :] % nx)).reshape(-1)
        st = poly.init(cfg, s.rho[idx], s.u[:, idx], s.T[idx])
        poly.step(st, 3)
        r, uu, t = poly.macros(cfg, st.f, st.g)
        k = 9 * 19 + 9
        assert abs(rho[c] - r[k]) <= TOL * r[k], (c, rho[c], r[k])
        assert abs(T[c] - t[k]) <= TOL * t[k], (c, T[c], t[k])
        cs = np.sqrt(s.gamma * t[k])
        assert np.abs(u[:, c] - uu[:, k]).max() <= TOL * max(np.abs(uu[:, k]).max(), cs), c
