"""The debug canary zones around a lattice's device buffers (Lattice(debug=True)), checked on
host tensors: writes inside the buffer keep the canaries, writes just outside are caught."""
import pytest
import torch


@pytest.fixture(scope="module")
def lat():
    from paper_1910_13515_gb300 import build
    build.build()
    from paper_1910_13515_gb300 import lattice
    return lattice


def test_writes_inside_keep_the_canaries(lat):
    g = lat.Guarded(1000, "cpu")
    assert g.buf.numel() == 1000 and g.intact()
    g.buf.fill_(3.0)
    g.buf[0] = float("nan")
    g.buf[-1] = -1.0
    assert g.intact()
    assert (g.buf.data_ptr() - g.full.data_ptr()) % 256 == 0  # alignment kept


@pytest.mark.parametrize("where", ["before", "after"])
def test_a_write_outside_is_caught(lat, where):
    pop, aux, guards = lat._buffers(8 * 500, 8 * 70, "cpu", debug=True)
    assert pop.numel() == 500 and aux.numel() == 70
    lat._check_guards(guards, "step")
    g = guards[1]
    k = g.PAD - 1 if where == "before" else g.PAD + g.buf.numel()
    g.full[k] = 0.0
    with pytest.raises(RuntimeError, match="auxiliary"):
        lat._check_guards(guards, "step")


def test_no_guards_without_debug(lat):
    pop, aux, guards = lat._buffers(800, 80, "cpu", debug=False)
    assert guards is None and pop.numel() == 100 and aux.numel() == 10
    lat._check_guards(None, "step")
