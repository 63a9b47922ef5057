"""Host-side failure detection on the GPU, with no device fault provoked: the bounded host wait
of lbm39_sync gives up with LBM39_ERR_TIMEOUT while work is still queued and leaves the lattice
usable and its state intact; the debug canary zones around a lattice's device buffers stay
intact over runs with every boundary kind and both precisions."""
import numpy as np
import pytest

from paper_1910_13515_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_1910_13515_gb300 import build
    build.build()
    from paper_1910_13515_gb300 import lbm39 as C
    from paper_1910_13515_gb300.lattice import Lattice
    return C, Lattice


def test_sync_timeout_is_reported_and_the_state_is_intact(mods):
    """30 queued steps of a 590k-cell box take tens of milliseconds; a 1 us limit on the host
    wait must run out (LBM39_ERR_TIMEOUT, the wait is a host poll of an event).  A later
    unbounded wait returns LBM39_OK, and the state equals that of a lattice whose wait was never
    cut short, bit for bit."""
    C, Lattice = mods
    s = inputs.box(seed=3, shape=(64, 96, 96), mach_rms=0.5)
    La, Lb = Lattice.from_setup(s), Lattice.from_setup(s)
    La.step(30)
    rc, failed = C.lbm39_sync(La.h, 1)
    assert rc == C.LBM39_ERR_TIMEOUT, C.lbm39_strerror(rc)
    rc, failed = C.lbm39_sync(La.h, -1)
    assert rc == C.LBM39_OK and failed == 0
    Lb.step(30)
    assert Lb.sync() == 0
    for x, y in zip(La.read_numpy(), Lb.read_numpy()):
        assert np.array_equal(x, y)
    La.step(2)  # the lattice stays usable after a timed-out wait
    assert La.sync() == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_canaries_stay_intact_on_the_airfoil(mods, precision):
    """Lattice(debug=True) puts 64 KiB canary zones before and after the population and
    auxiliary buffers and checks them after init and every step (raising on a change).  The
    small airfoil (bounce-back, freestream, outflow cells, both AA parities, fill kernels) runs
    40 steps clean, and its result equals the unguarded run bit for bit."""
    C, Lattice = mods
    s = inputs.naca(nx=96, ny=48, chord=24, x_le=24)
    Ld = Lattice.from_setup(s, precision=precision, debug=True)
    for _ in range(40):
        Ld.step(1)
    assert Ld.sync() == 0
    assert all(g.intact() for g in Ld._guards)
    L = Lattice.from_setup(s, precision=precision)
    L.step(40)
    assert L.sync() == 0
    for x, y in zip(Ld.read_numpy(), L.read_numpy()):
        assert np.array_equal(x, y)
