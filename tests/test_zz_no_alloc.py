"""lbm39_conserved_noalloc: the conserved sums for callers that cannot allocate device
memory (its scratch is a fixed array inside the library).  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_sums_match_stats_on_two_calls_in_a_row():
    from paper_1910_13515_gb300 import build
    build.build()
    from paper_1910_13515_gb300 import inputs
    from paper_1910_13515_gb300 import lbm39 as C
    from paper_1910_13515_gb300.lattice import Lattice

    for s, prec in ((inputs.box(seed=8, shape=(20, 18, 16)), C.LBM39_FP64),
                    (inputs.naca(nx=96, ny=48, chord=24, x_le=24), C.LBM39_FP64),
                    (inputs.box(seed=9, shape=(12, 12, 12)), C.LBM39_MIXED)):
        L = Lattice.from_setup(s, precision=prec)
        for steps in (3, 4):  # two calls in a row, at both AA parities
            L.step(steps)
            assert L.sync() == 0
            want = np.array(L.stats().conserved)
            got = np.full(5, np.nan)
            rc = C.lbm39_conserved_noalloc(L.h, got.ctypes.data_as(ctypes.c_void_p))
            assert rc == C.LBM39_OK, C.lbm39_strerror(rc)
            scale = np.array([abs(want[0])] * 4 + [abs(want[4])])
            assert np.all(np.abs(got - want) <= 1e-12 * scale), (got, want)


def test_noalloc_rejects_bad_arguments():
    from paper_1910_13515_gb300 import lbm39 as C
    out = np.zeros(5)
    assert C.lbm39_conserved_noalloc(None, out.ctypes.data_as(ctypes.c_void_p)) == C.LBM39_ERR_ARG
