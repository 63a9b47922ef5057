"""The chord-Newton hybrid root finder (lbm39_params.root_finder = 1) on the GPU against the
oracle's hybrid (oracle39.c o39_newton_hybrid), through the C ABI: FP64 parity to 1e-11 in
rho/u/T on the full 13-constraint solve and the z-mirror reduced one, the same Newton-update
counts, and the same flow as the Newton root finder (both solve every cell below the same
residual)."""
import numpy as np
import pytest

from gpu_helpers import TOL, rel_diffs, run_oracle
from oracle import oracle39 as o
from paper_1910_13515_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_1910_13515_gb300 import build
    build.build()
    from paper_1910_13515_gb300 import lbm39 as C
    from paper_1910_13515_gb300.lattice import Lattice
    return C, Lattice


CASES = {
    "box16": (lambda: inputs.box(seed=0, shape=(16, 16, 16)), 100),
    "box_ragged_ma08": (lambda: inputs.box(seed=1, shape=(9, 11, 13)), 8),
    "sod": (lambda: inputs.sod(400), 160),
    "naca_small_reduced": (lambda: inputs.naca(nx=96, ny=48, chord=24, x_le=24), 100),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_chord_newton_parity(mods, case):
    C, Lattice = mods
    make, n = CASES[case]
    s = make()
    L = Lattice.from_setup(s, root_finder=1)
    L.step(n)
    assert L.sync() == 0
    st, fo = run_oracle(s, n, root_finder=1)
    assert fo == 0
    d = rel_diffs(L.read_numpy(), o.macros(st), s.mask, s.gamma)
    assert max(d) <= TOL, d
    gs = L.stats()
    assert abs(gs.newton_updates - st.stats.newton_updates) <= 1e-3 * st.stats.newton_updates + 2
    # the same equilibria as Newton-Raphson: the Newton oracle run agrees too
    st0, _ = run_oracle(s, n)
    assert max(rel_diffs(L.read_numpy(), o.macros(st0), s.mask, s.gamma)) <= TOL


def test_chord_newton_only_for_fp64_pr1(mods):
    C, Lattice = mods
    from paper_1910_13515_gb300.lattice import params_from_setup
    s = inputs.box(seed=2, shape=(4, 4, 4))
    for over in ({"root_finder": 1, "precision": 1}, {"root_finder": 1, "prandtl": 0.71},
                 {"root_finder": 2}):
        rc, _, _ = C.lbm39_query_bytes(params_from_setup(s, **over))
        assert rc == C.LBM39_ERR_ARG, over
