"""The Python calls the README documents exist with the documented parameters (no GPU)."""
import inspect

import pytest


@pytest.fixture(scope="module")
def pkg():
    from paper_1910_13515_gb300 import build
    build.build()
    from paper_1910_13515_gb300 import diagnostics, inputs, lattice, lbm39
    return lattice, diagnostics, inputs, lbm39


def test_documented_calls_exist(pkg):
    lattice, diagnostics, inputs, C = pkg
    for name in ("from_setup", "init", "init_host", "step", "sync", "read", "read_numpy",
                 "read_host", "diag_fields", "stats", "checkpoint", "restore", "close"):
        assert callable(getattr(lattice.Lattice, name)), name
    for name in ("init", "step", "read", "read_numpy", "conserved", "close"):
        assert callable(getattr(lattice.PolyLattice, name)), name
    assert "debug" in inspect.signature(lattice.Lattice.from_setup).parameters
    assert "precision" in inspect.signature(lattice.Lattice.from_setup).parameters
    assert {"nx", "ny", "nz", "gamma", "tau", "debug"} <= set(
        inspect.signature(lattice.PolyLattice).parameters)
    assert callable(diagnostics.surface_cp) and callable(inputs.subsonic_box)
    assert C.LBM39_MIXED != C.LBM39_FP64


def test_precision_form_reference_follows_the_far_field(pkg):
    """Lattice's parameters for the precision form: deviations from the far-field equilibrium on
    a lattice with freestream cells, from the library's rest reference otherwise; FP64 lattices
    and explicit overrides are left alone, and the library accepts both."""
    lattice, _, inputs, C = pkg
    naca = inputs.naca(nx=96, ny=48, chord=24, x_le=24)
    p = lattice.params_from_setup(naca, C.LBM39_MIXED)
    assert (p.ref_rho, list(p.ref_u), p.ref_T) == (naca.rho_inf, [naca.u_inf[0], 0.0, 0.0],
                                                   naca.T_inf)
    assert C.lbm39_query_bytes(p)[0] == 0
    p = lattice.params_from_setup(naca, C.LBM39_FP64)
    assert list(p.ref_u) == [0.0, 0.0, 0.0]
    p = lattice.params_from_setup(naca, C.LBM39_MIXED, ref_u=(0.0, 0.0, 0.0), ref_T=0.6)
    assert list(p.ref_u) == [0.0, 0.0, 0.0] and p.ref_T == 0.6
    for s in (inputs.box(n=8, seed=1, shape=(4, 5, 6)), inputs.sod(400)):
        p = lattice.params_from_setup(s, C.LBM39_MIXED)
        assert (p.ref_rho, list(p.ref_u), p.ref_T) == (1.0, [0.0, 0.0, 0.0], 0.5)
