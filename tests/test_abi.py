"""Host-only checks of the C ABI: the library builds, loads and exports every symbol that
include/*.h declares; argument validation that happens before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def C():
    from paper_1910_13515_gb300 import build
    build.build()
    from paper_1910_13515_gb300 import lbm39
    return lbm39


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm39_\w+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(C):
    names = declared_functions()
    assert "lbm39_step" in names and "lbm39_create" in names and len(names) >= 16
    assert "lbm39_poly_step" in names and "lbm39_poly_create" in names
    lib = ctypes.CDLL(C.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def test_velocity_table_matches_the_paper_set_and_oracle(C, oracle):
    vel = np.zeros((39, 3), np.int32)
    w = np.zeros(39)
    assert C.lbm39_velocities(vel.ctypes.data, w.ctypes.data) == 0
    ov, ow, oopp = oracle.lattice()
    lib_map = {tuple(v): wi for v, wi in zip(vel, w)}
    orc_map = {tuple(v): wi for v, wi in zip(ov, ow)}
    assert lib_map.keys() == orc_map.keys()
    for k in lib_map:
        assert lib_map[k] == orc_map[k]
    # rest velocity first, then (xi, -xi) pairs
    assert tuple(vel[0]) == (0, 0, 0)
    for i in range(1, 39, 2):
        assert np.array_equal(vel[i], -vel[i + 1])


def test_default_params_and_sizes(C):
    p = C.lbm39_default_params(10, 8, 6)
    assert (p.nx, p.ny, p.nz) == (10, 8, 6) and list(p.periodic) == [1, 1, 1]
    assert p.gamma == 1.4 and p.newton_tol == 1e-12 and p.newton_min_upd == 0
    rc, pop_b, aux_b = C.lbm39_query_bytes(p)
    assert rc == 0
    N = 480
    Np = (N + 63) // 64 * 64
    assert pop_b == 78 * 8 * Np
    assert aux_b >= 52 * 8 * Np


def test_params_layout_matches_the_header(C):
    """lbm39_default_params writes exactly the binding's lbm39_params: nothing past its end
    (the C struct is no larger), and the last field (ref_u) at the binding's offset."""
    import ctypes
    n = ctypes.sizeof(C.lbm39_params)
    buf = (ctypes.c_ubyte * (n + 64))(*([0xAB] * (n + 64)))
    C._lib.lbm39_default_params(ctypes.cast(buf, ctypes.POINTER(C.lbm39_params)), 8, 8, 8)
    assert bytes(buf[n:]) == b"\xab" * 64
    p = C.lbm39_params.from_buffer(buf)
    assert list(p.ref_u) == [0.0, 0.0, 0.0] and p.ref_T == 0.5 and p.prandtl == 1.0
    assert p.root_finder == 0 and (p.nx, p.ny, p.nz) == (8, 8, 8)


def test_nonfinite_reference_velocity_rejected(C):
    p = C.lbm39_default_params(8, 8, 8)
    p.precision = C.LBM39_MIXED
    p.ref_u[0] = float("nan")
    assert C.lbm39_query_bytes(p)[0] == C.LBM39_ERR_ARG
    p.ref_u[0] = 1.0
    assert C.lbm39_query_bytes(p)[0] == 0


@pytest.mark.parametrize("field,value", [("nx", 0), ("gamma", 1.0), ("tau", 0.4),
                                         ("newton_tol", 0.0), ("newton_maxit", 0),
                                         ("precision", 7)])
def test_bad_params_rejected(C, field, value):
    p = C.lbm39_default_params(8, 8, 8)
    setattr(p, field, value)
    rc, _, _ = C.lbm39_query_bytes(p)
    assert rc == C.LBM39_ERR_ARG


def test_create_validation_before_any_gpu_call(C):
    p = C.lbm39_default_params(8, 8, 8)
    vel = np.zeros((39, 3), np.int32)
    C.lbm39_velocities(vel.ctypes.data, None)
    bad = vel.copy()
    bad[[1, 2]] = bad[[2, 1]]
    fake = 1 << 20  # never dereferenced: validation fails first
    rc, h = C.lbm39_create(p, bad.ctypes.data, None, fake, fake, None, None)
    assert rc == C.LBM39_ERR_LATTICE and not h
    rc, h = C.lbm39_create(p, vel.ctypes.data, None, fake + 8, fake, None, None)
    assert rc == C.LBM39_ERR_ARG  # misaligned buffer
    p.periodic[0] = 0
    rc, h = C.lbm39_create(p, vel.ctypes.data, None, fake, fake, None, None)
    assert rc == C.LBM39_ERR_MASK  # non-periodic axis needs a mask


def test_null_handles_and_strerror(C):
    assert C.lbm39_step(None, 1) == C.LBM39_ERR_ARG
    assert C.lbm39_sync(None, 0)[0] == C.LBM39_ERR_ARG
    assert C.lbm39_read(None, None, None, None, None) == C.LBM39_ERR_ARG
    assert C.lbm39_checkpoint_bytes(None) == 0
    C.lbm39_destroy(None)
    for code in range(-7, 1):
        assert C.lbm39_strerror(code) != "unknown status"
    assert C.lbm39_strerror(-99) == "unknown status"


def poly_params(C, nx=16, ny=8, nz=4):
    p = C.lbm39_default_params(nx, ny, nz)
    p.kn_sensor = 0
    return p


@pytest.mark.parametrize("field,value", [("kn_sensor", 1), ("precision", 1), ("tau", 0.49),
                                         ("gamma", 1.0), ("nx", 0)])
def test_poly_bad_params_rejected(C, field, value):
    p = poly_params(C)
    setattr(p, field, value)
    assert C.lbm39_poly_query_bytes(p)[0] == C.LBM39_ERR_ARG


def test_poly_sizes_and_state_checks_before_any_gpu_call(C):
    p = poly_params(C, 10, 7, 3)
    rc, pop, aux = C.lbm39_poly_query_bytes(p)
    assert rc == C.LBM39_OK
    assert pop == 8 * 78 * 256  # 210 cells, plane stride rounded up to 64
    assert aux >= 8 * 5 * 1024
    for a in range(3):  # every axis must be periodic
        q = poly_params(C, 10, 7, 3)
        q.periodic[a] = 0
        assert C.lbm39_poly_query_bytes(q)[0] == C.LBM39_ERR_ARG
    big = poly_params(C, 2048, 2048, 512)  # 2^31 cells
    assert C.lbm39_poly_query_bytes(big)[0] == C.LBM39_ERR_ARG
    fake = 1 << 20  # never dereferenced: create does no device work
    assert C.lbm39_poly_create(p, fake + 8, fake, None)[0] == C.LBM39_ERR_ARG
    rc, h = C.lbm39_poly_create(p, fake, fake, None)
    assert rc == C.LBM39_OK and h
    try:
        assert C.lbm39_poly_time(h) == 0
        assert C.lbm39_poly_step(h, 1) == C.LBM39_ERR_STATE
        assert C.lbm39_poly_step(h, -1) == C.LBM39_ERR_ARG
        assert C.lbm39_poly_read(h, None, None, None, None) == C.LBM39_ERR_STATE
        s = np.zeros(5)
        assert C.lbm39_poly_conserved(h, s.ctypes.data) == C.LBM39_ERR_STATE
        assert C.lbm39_poly_init(h, None, None, None) == C.LBM39_ERR_ARG
    finally:
        C.lbm39_poly_destroy(h)
    assert C.lbm39_poly_time(None) == -1
    assert C.lbm39_poly_step(None, 1) == C.LBM39_ERR_ARG
    C.lbm39_poly_destroy(None)
