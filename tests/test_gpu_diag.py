"""Per-cell diagnostic fields (lbm39_diag_fields): the Knudsen sensor eps and the Newton-update
count of the next step (the paper's sensor and iteration maps, Sec. 4), against the oracle's
per-cell collision on the oracle's own state at the same time, and the state left unchanged.

The update count is an integer decided by FP64 stopping tests (the 1e-12 tolerance and the
1e-14 warm-start test) on both sides.  A residual within rounding of a threshold flips the
count by one: perturbing the oracle's own state by a relative 1e-15 flips 0.24% of the counts
on the 40-step small airfoil, always by +-1 (measured on the CPU).  So counts may differ by
exactly one in at most 2% of the cells, failures (-1) must agree exactly, and eps is compared
where the counts agree, cell by cell to 1e-10 + 1e-9 |eps| (the same perturbation moves eps
by up to 1.1e-10 relative; eps reaches 1e4 where f^eq is tiny)."""
import numpy as np
import pytest

from gpu_helpers import oracle_cfg
from oracle import oracle39 as o
from paper_1910_13515_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Lat():
    from paper_1910_13515_gb300 import build
    build.build()
    from paper_1910_13515_gb300.lattice import Lattice
    return Lattice


def oracle_fields(s, st):
    """(eps, n_upd) of the oracle state st: one collision per fluid cell on copies, with the
    cell's fallback flag and the state's time step; -1 where the solve fails."""
    cfg = oracle_cfg(s)
    eps = np.zeros(s.ncells)
    nupd = np.zeros(s.ncells, np.int64)
    for c in np.flatnonzero(s.mask == 0):
        _, _, _, nu, e, _, status, _ = o.collide_cell(cfg, st.f[c], st.g[c], st.lam[c],
                                                      on_fallback=bool(st.on_fb[c]), t=st.t)
        eps[c] = e
        nupd[c] = -1 if status else nu
    return eps, nupd


def gpu_fields(L):
    eps, nupd = L.diag_fields()
    L.stream.synchronize()
    return eps.cpu().numpy(), nupd.cpu().numpy().astype(np.int64)


def compare(s, L, st):
    ge, gn = gpu_fields(L)
    oe, on = oracle_fields(s, st)
    fl = s.mask == 0
    same = (gn == on) & fl
    assert np.array_equal(gn[fl] == -1, on[fl] == -1)
    flips = gn[fl] != on[fl]
    assert flips.sum() <= max(1, int(0.02 * fl.sum())), flips.sum()
    assert (np.abs(gn[fl] - on[fl])[flips] == 1).all()
    assert np.all(np.abs(ge[same] - oe[same]) <= 1e-10 + 1e-9 * np.abs(oe[same]))
    assert (ge[~fl] == 0).all() and (gn[~fl] == 0).all()
    return ge, gn


@pytest.mark.parametrize("nsteps", [0, 1, 40])
def test_fields_match_oracle_on_the_small_airfoil(Lat, nsteps):
    """Masks, freestream and outflow cells, the z-mirror (nine-constraint) path, both parities."""
    s = inputs.naca(nx=96, ny=48, chord=24, x_le=24)
    L = Lat.from_setup(s)
    L.step(nsteps)
    L.sync()
    st = o.init(oracle_cfg(s), s.mask, s.rho, s.u, s.T)
    o.step(st, nsteps)
    ge, gn = compare(s, L, st)
    if nsteps == 40:
        assert ge[s.mask == 0].max() > 1e-3  # the bow shock departs from equilibrium


def test_fields_match_oracle_on_a_box_full_solve(Lat):
    s = inputs.box(seed=1, shape=(9, 11, 13))
    L = Lat.from_setup(s)
    L.step(7)
    L.sync()
    st = o.init(oracle_cfg(s), s.mask, s.rho, s.u, s.T)
    o.step(st, 7)
    _, gn = compare(s, L, st)
    assert gn.max() >= 2


def test_cells_outside_the_cone_read_minus_one(Lat):
    s = inputs.uniform(12, 10, 8, u=(1.0, 0.2, 0.0), T=0.5, tau=0.6)
    blob = np.zeros((8, 10, 12), bool)
    blob[3:5, 4:7, 5:8] = True
    b = blob.reshape(-1)
    s.u, s.T, s.rho = s.u.copy(), s.T.copy(), s.rho.copy()
    s.u[0, b], s.u[1, b], s.T[b], s.rho[b] = 1.416, -0.348, 0.414, 0.954
    L = Lat.from_setup(s)
    L.step(2)
    L.sync()
    st = o.init(oracle_cfg(s), s.mask, s.rho, s.u, s.T, allow_failed=True)
    o.step(st, 2)
    _, gn = compare(s, L, st)
    assert (gn[b] == -1).all() and (gn[~b] >= 0).all()


def test_fields_leave_the_state_unchanged(Lat):
    s = inputs.box(seed=3, shape=(8, 8, 8))
    L = Lat.from_setup(s)
    L.step(3)
    L.sync()
    s0 = L.stats()
    L.diag_fields()
    L.sync()
    s1 = L.stats()
    assert s1.newton_updates == s0.newton_updates and s1.failed_cells == s0.failed_cells
    assert s1.time == s0.time == 3
    buf = L.checkpoint()
    L.diag_fields()
    L.step(4)
    a = L.read_numpy()
    L.restore(buf)
    L.step(4)
    b = L.read_numpy()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_precision_form_fields_are_close_to_fp64(Lat):
    from paper_1910_13515_gb300 import lbm39 as C
    s = inputs.box(seed=2, shape=(10, 9, 8), mach_rms=0.4)
    Lf = Lat.from_setup(s)
    Lm = Lat.from_setup(s, precision=C.LBM39_MIXED, ref_rho=1.0, ref_T=0.5)
    Lf.step(2)
    Lm.step(2)
    Lf.sync()
    Lm.sync()
    ef, nf = gpu_fields(Lf)
    em, nm = gpu_fields(Lm)
    assert np.isfinite(em).all() and (nm >= 0).all()
    np.testing.assert_allclose(em, ef, rtol=1e-3, atol=1e-6)


@pytest.mark.parametrize("root_finder,precision", [(0, 0), (1, 0), (2, 0), (3, 0), (0, 1)])
def test_update_counts_are_those_the_next_step_takes(Lat, root_finder, precision):
    """The n_upd field does the next step's solve with the lattice's root finder (the precision
    form: its single-precision start and FP32 direction): summed over the cells it equals the
    Newton updates that step adds to the counters, and its -1 cells are the step's failures."""
    s = inputs.box(seed=4, shape=(12, 10, 9))
    L = Lat.from_setup(s, root_finder=root_finder, precision=precision)
    L.step(3)
    L.sync()
    _, gn = gpu_fields(L)
    s0 = L.stats()
    L.step(1)
    L.sync()
    s1 = L.stats()
    assert gn[gn >= 0].sum() == s1.newton_updates - s0.newton_updates
    assert (gn == -1).sum() == s1.failed_cells - s0.failed_cells
