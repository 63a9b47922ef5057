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
