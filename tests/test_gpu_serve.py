"""Serving form on the GPU: requests run together through packed, graph-replayed steps give
exactly (bit for bit) what each gives alone through lbm39_step, and the served FP64 results
match the FP64 CPU oracle."""
import numpy as np
import pytest

from paper_1910_13515_gb300 import inputs

pytestmark = pytest.mark.gpu


def small_requests(n=10, seed=7):
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    for rid in range(n):
        t += rng.exponential(0.005)
        steps = int(rng.integers(20, 70))
        if rid % 2 == 0:
            s = inputs.random_riemann(rng, 200, 600, steps=steps)
        else:
            s = inputs.shear_layer(int(rng.choice([16, 24, 32])), float(rng.uniform(0.5, 2.0)),
                                   steps=steps, seed=rid)
        reqs.append(inputs.Request(rid, t, s))
    return reqs


@pytest.mark.parametrize("precision", [0, 1])
def test_served_results_equal_results_alone(precision):
    from paper_1910_13515_gb300 import build
    build.build()
    from paper_1910_13515_gb300.lattice import Lattice
    from paper_1910_13515_gb300.serve import GpuBackend, Scheduler

    reqs = small_requests()
    be = GpuBackend(precision=precision, max_lattices=8, max_cells=1 << 16, graph_steps=8)
    one = max(be.bytes_for(r.setup) for r in reqs)
    rep = Scheduler(be, budget_bytes=3 * one, max_resident=4, chunk_steps=20).run(reqs)
    be.close()
    assert rep.max_resident >= 2  # the mix really ran together
    assert sorted(rep.results) == [r.rid for r in reqs]
    for r in reqs:
        L = Lattice.from_setup(r.setup, precision=precision)
        L.step(r.setup.steps)
        assert L.sync() == 0
        alone = L.read_numpy()
        mixed = rep.results[r.rid]
        for a, b in zip(alone, mixed):
            assert np.array_equal(a, b), r.rid
    assert rep.p99_ms >= rep.p50_ms > 0 and rep.mlups > 0


def test_served_results_match_the_oracle():
    """Served FP64 results against the FP64 CPU oracle run of each request alone (1e-11 in
    rho/u/T): Riemann tubes (outflow ends, tau = 1/2 with the sensor) and doubly periodic shear
    layers, packed together and admitted while other requests run."""
    from paper_1910_13515_gb300 import build
    build.build()
    from gpu_helpers import TOL, rel_diffs, run_oracle
    from oracle import oracle39 as o
    from paper_1910_13515_gb300.serve import GpuBackend, Scheduler

    reqs = small_requests(8, seed=11)
    kinds = {r.setup.name.split("_")[0] for r in reqs}
    assert kinds == {"riemann", "shear"}
    be = GpuBackend(precision=0, max_lattices=8, max_cells=1 << 16, graph_steps=8)
    one = max(be.bytes_for(r.setup) for r in reqs)
    rep = Scheduler(be, budget_bytes=3 * one, max_resident=4, chunk_steps=16).run(reqs)
    be.close()
    assert rep.max_resident >= 2
    for r in reqs:
        st, failed = run_oracle(r.setup, r.setup.steps)
        assert failed == 0
        d = rel_diffs(rep.results[r.rid], o.macros(st), r.setup.mask, r.setup.gamma)
        assert max(d) <= TOL, (r.setup.name, d)


def test_packed_mix_of_constraint_systems():
    """A batch that holds lattices of both constraint systems -- one-cell-thick shear layers and
    tubes (the nine-constraint z-mirror solve) and 3-D boxes (all 13) -- runs each set with its
    own packed instantiation; every result equals the lattice run alone, bit for bit."""
    from paper_1910_13515_gb300 import build
    build.build()
    from paper_1910_13515_gb300.lattice import Lattice
    from paper_1910_13515_gb300.serve import GpuBackend, Scheduler

    rng = np.random.default_rng(23)
    reqs = []
    for rid in range(6):
        steps = int(rng.integers(10, 30))
        if rid % 3 == 0:
            s = inputs.box(seed=rid, shape=(6, 7, 9), steps=steps, mach_rms=0.5)
        elif rid % 3 == 1:
            s = inputs.shear_layer(16, 1.2, steps=steps, seed=rid)
        else:
            s = inputs.random_riemann(rng, 200, 300, steps=steps)
        reqs.append(inputs.Request(rid, 0.001 * rid, s))
    be = GpuBackend(precision=0, max_lattices=8, max_cells=1 << 16, graph_steps=4)
    rep = Scheduler(be, budget_bytes=1 << 34, max_resident=8, chunk_steps=8).run(reqs)
    be.close()
    assert rep.max_resident >= 3
    for r in reqs:
        L = Lattice.from_setup(r.setup)
        L.step(r.setup.steps)
        assert L.sync() == 0
        for a, b in zip(L.read_numpy(), rep.results[r.rid]):
            assert np.array_equal(a, b), r.setup.name
