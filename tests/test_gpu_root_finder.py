"""The other root finders of the constraint equations on the GPU against the oracle's
(lbm39_params.root_finder 1: the chord-Newton hybrid, oracle39.c o39_newton_hybrid; 2: Newton with
a single-precision direction, o39_newton_fp32dir; 3: that after a single-precision start,
o39_newton_fp32start), through the C ABI: FP64 parity to 1e-11 in
rho/u/T on the full 13-constraint solve and the z-mirror reduced one, the Newton-update counts,
and the same flow as the Newton root finder (all solve every cell below the same residual)."""
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


@pytest.mark.parametrize("solver", [1, 2, 3])
@pytest.mark.parametrize("case", sorted(CASES))
def test_root_finder_parity(mods, case, solver):
    C, Lattice = mods
    make, n = CASES[case]
    s = make()
    L = Lattice.from_setup(s, root_finder=solver)
    L.step(n)
    assert L.sync() == 0
    st, fo = run_oracle(s, n, root_finder=solver)
    assert fo == 0
    d = rel_diffs(L.read_numpy(), o.macros(st), s.mask, s.gamma)
    assert max(d) <= TOL, d
    gs = L.stats()
    # the kernel decides with the residual of the nine-constraint system on the z-mirror
    # reduced lattice (the oracle always solves all 13), and solver 2 forms its direction in
    # FP32 with another summation and factorisation than the oracle's: a few cells take one
    # update more or less (measured: 0.14% and 2.8% on the small airfoil); solver 3's float
    # start (CUDA's expf and the generated sums against the oracle's loops) likewise
    slack = 5e-3 if solver == 1 else 5e-2
    assert abs(gs.newton_updates - st.stats.newton_updates) <= slack * st.stats.newton_updates + 2
    if solver == 3:
        assert gs.start32_updates >= gs.start32_solves > 0
        assert gs.start32_updates <= 4 * gs.start32_solves
        st2, _ = run_oracle(s, n, root_finder=2)
        # the start saves FP64 updates (oracle: 0.56-0.69 of solver 2's on these cases)
        assert gs.newton_updates <= 0.8 * st2.stats.newton_updates
    else:
        assert gs.start32_updates == gs.start32_solves == 0
    # the same equilibria as Newton-Raphson: the Newton oracle run agrees too
    st0, _ = run_oracle(s, n)
    assert max(rel_diffs(L.read_numpy(), o.macros(st0), s.mask, s.gamma)) <= TOL


def test_other_root_finders_only_for_fp64_pr1(mods):
    C, Lattice = mods
    from paper_1910_13515_gb300.lattice import params_from_setup
    s = inputs.box(seed=2, shape=(4, 4, 4))
    for over in ({"root_finder": 1, "precision": 1}, {"root_finder": 1, "prandtl": 0.71},
                 {"root_finder": 2, "precision": 1}, {"root_finder": 3, "precision": 1},
                 {"root_finder": 3, "prandtl": 2.0}, {"root_finder": 4}, {"root_finder": -1}):
        rc, _, _ = C.lbm39_query_bytes(params_from_setup(s, **over))
        assert rc == C.LBM39_ERR_ARG, over
