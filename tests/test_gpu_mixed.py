"""The precision form (FP32 deviation storage, FP32 collision, FP64 moments and constraint
solve) against the FP64 oracle and the FP64 CUDA path, through the C ABI.

Bars: L1 relative error in rho, u, T against the FP64 oracle <= 1e-4; mass, momentum and
energy drift stated per 1000 steps."""
import numpy as np
import pytest

from gpu_helpers import rel_diffs, run_oracle
from oracle import oracle39 as o
from paper_1910_13515_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mod():
    from paper_1910_13515_gb300 import build
    build.build()
    from paper_1910_13515_gb300 import lbm39 as C
    from paper_1910_13515_gb300.lattice import Lattice
    return C, Lattice


def l1_rel(a, b, mask):
    fl = mask == 0
    ra, ua, Ta = a[:3]
    rb, ub, Tb = b[:3]
    return (np.abs(ra[fl] - rb[fl]).mean() / np.abs(rb[fl]).mean(),
            np.abs(ua[:, fl] - ub[:, fl]).mean() / np.sqrt((ub[:, fl] ** 2).sum(0)).mean(),
            np.abs(Ta[fl] - Tb[fl]).mean() / np.abs(Tb[fl]).mean())


@pytest.mark.parametrize("shape,seed,steps", [((16, 16, 16), 0, 100), ((12, 10, 9), 3, 60)])
def test_mixed_box_l1_error_vs_oracle(mod, shape, seed, steps):
    C, Lattice = mod
    s = inputs.box(seed=seed, shape=shape)
    L = Lattice.from_setup(s, precision=C.LBM39_MIXED)
    L.step(steps)
    assert L.sync() == 0
    g = L.read_numpy()
    st, fo = run_oracle(s, steps)
    err = l1_rel(g, o.macros(st), s.mask)
    assert max(err) <= 1e-4, err


@pytest.mark.parametrize("reference,bar", [("far field", 1e-4), ("rest", 2e-3)])
def test_mixed_naca_small_l1_error_vs_oracle(mod, reference, bar):
    """Impulsive start of Ma 1.5 flow on a 24-cell chord, against the FP64 oracle.

    Far-field reference (the default for a lattice with freestream cells): the stored FP32
    values are deviations from the far-field equilibrium, zero in the undisturbed flow and of
    the size of the populations themselves near the airfoil, so FP32 resolves them to ~6e-8
    of the population.  Held to the precision form's 1e-4 after 100 steps (storage rounding
    emulated on the oracle gives 5.9e-5).

    Rest reference (ref_u = 0): at Ma 1.5 the smallest populations lie four to five orders of
    magnitude below their reference values, so their deviations are stored to ~1e-3 of the
    populations; that moves eps of cells near a threshold of Eq. (alpha) across it, and each
    flip changes tau_eff by 5-35% in that cell.  Before the first flip (steps 0-2) the forms
    agree to ~1e-8; after 100 steps the L1 difference is ~6e-4, held to 2e-3."""
    C, Lattice = mod
    s = inputs.naca(nx=96, ny=48, chord=24, x_le=24)
    over = {} if reference == "far field" else {"ref_u": (0.0, 0.0, 0.0)}
    L = Lattice.from_setup(s, precision=C.LBM39_MIXED, **over)
    assert list(L.params.ref_u) == ([s.u_inf[0], 0.0, 0.0] if not over else [0.0, 0.0, 0.0])
    L.step(2)
    assert L.sync() == 0
    st, fo = run_oracle(s, 2)
    assert max(l1_rel(L.read_numpy(), o.macros(st), s.mask)) <= 1e-6
    L.step(98)
    assert L.sync() == 0
    o.step(st, 98)
    err = l1_rel(L.read_numpy(), o.macros(st), s.mask)
    print(f"precision form, {reference} reference: L1 after 100 steps {err}")
    assert max(err) <= bar, err


def test_mixed_sod_l1_error_vs_oracle(mod):
    C, Lattice = mod
    s = inputs.sod(400)
    L = Lattice.from_setup(s, precision=C.LBM39_MIXED)
    L.step(160)
    assert L.sync() == 0
    st, fo = run_oracle(s, 160)
    err = l1_rel(L.read_numpy(), o.macros(st), s.mask)
    assert max(err) <= 1e-4, err


def test_mixed_obstacle_box_l1_error_vs_oracle(mod):
    """Solid block across the periodic boundary: bounce-back in the precision form."""
    C, Lattice = mod
    s = inputs.box(seed=5, shape=(7, 10, 12))
    s.mask.reshape(7, 10, 12)[2:4, 3:6, [10, 11, 0]] = 1
    L = Lattice.from_setup(s, precision=C.LBM39_MIXED)
    L.step(60)
    assert L.sync() == 0
    st, fo = run_oracle(s, 60)
    err = l1_rel(L.read_numpy(), o.macros(st), s.mask)
    assert max(err) <= 1e-4, err


def test_mixed_conservation_drift(mod):
    """Periodic box, 1000 steps: relative drift of mass and energy and momentum drift
    relative to the mass (all FP64 sums of the stored state)."""
    C, Lattice = mod
    s = inputs.box(seed=2, shape=(16, 16, 16))
    L = Lattice.from_setup(s, precision=C.LBM39_MIXED)
    c0 = np.array(L.stats().conserved)
    L.step(1000)
    assert L.sync() == 0
    c1 = np.array(L.stats().conserved)
    drift = np.abs(c1 - c0) / np.array([c0[0]] * 4 + [c0[4]])
    assert drift.max() <= 1e-5, drift


def test_mixed_uniform_flow(mod):
    C, Lattice = mod
    s = inputs.uniform(6, 5, 4, u=(0.3, -0.2, 0.1), T=0.5)
    L = Lattice.from_setup(s, precision=C.LBM39_MIXED)
    L.step(200)
    assert L.sync() == 0
    rho, u, T, p = L.read_numpy()
    assert np.abs(rho - 1).max() < 1e-6 and np.abs(u[0] - 0.3).max() < 1e-6
    assert np.abs(T - 0.5).max() < 1e-6


def test_mixed_checkpoint_resume_is_bit_identical(mod):
    C, Lattice = mod
    s = inputs.box(seed=6, shape=(8, 8, 8))
    L = Lattice.from_setup(s, precision=C.LBM39_MIXED)
    L.step(5)
    buf = L.checkpoint()
    L.step(4)
    a = L.read_numpy()
    L.restore(buf)
    L.step(4)
    for x, y in zip(a, L.read_numpy()):
        assert np.array_equal(x, y)
