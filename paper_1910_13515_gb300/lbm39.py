"""Thin ctypes binding of the C ABI in include/lbm39.h (argument marshalling only).

Every function has the C name and argument order; pointers are passed as
integers (device pointers from torch tensors' ``data_ptr()``, host pointers
from numpy arrays' ``ctypes.data``).  Functions return the C status code;
``check`` turns a non-zero code into an exception.  Importing this module
loads liblbm39.so and raises if it has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm39.so")

Q = 39
NM = 13

LBM39_OK = 0
LBM39_ERR_ARG = -1
LBM39_ERR_CUDA = -2
LBM39_ERR_NEWTON = -3
LBM39_ERR_TIMEOUT = -4
LBM39_ERR_LATTICE = -5
LBM39_ERR_MASK = -6
LBM39_ERR_STATE = -7

LBM39_FP64 = 0
LBM39_MIXED = 1


class lbm39_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("periodic", ctypes.c_int32 * 3),
        ("gamma", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("kn_sensor", ctypes.c_int32),
        ("newton_tol", ctypes.c_double),
        ("newton_maxit", ctypes.c_int32),
        ("newton_min_upd", ctypes.c_int32),
        ("init_maxit", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("ref_rho", ctypes.c_double), ("ref_T", ctypes.c_double),
        ("rho_inf", ctypes.c_double), ("u_inf", ctypes.c_double * 3), ("T_inf", ctypes.c_double),
        ("reduce_2d", ctypes.c_int32),
        ("prandtl", ctypes.c_double),
        ("root_finder", ctypes.c_int32),
        ("ref_u", ctypes.c_double * 3),
    ]


class lbm39_stats_t(ctypes.Structure):
    _fields_ = [
        ("time", ctypes.c_int64),
        ("fluid_cells", ctypes.c_int64),
        ("failed_cells", ctypes.c_int64),
        ("newton_updates", ctypes.c_int64),
        ("newton_hist", ctypes.c_int64 * 32),
        ("eps_hist", ctypes.c_int64 * 4),
        ("conserved", ctypes.c_double * 5),
        ("start32_updates", ctypes.c_int64),
        ("start32_solves", ctypes.c_int64),
    ]


class LBM39Error(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {lbm39_strerror(code)} ({code})")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it with paper_1910_13515_gb300.build.build() "
            "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER(lbm39_params)
    vp, i, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    sig = {
        "lbm39_default_params": (None, [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
        "lbm39_velocities": (i, [vp, vp]),
        "lbm39_query_bytes": (i, [P, ctypes.POINTER(sz), ctypes.POINTER(sz)]),
        "lbm39_create": (i, [P, vp, vp, vp, vp, vp, vp, ctypes.POINTER(vp)]),
        "lbm39_init": (i, [vp, vp, vp, vp]),
        "lbm39_init_host": (i, [vp, vp, vp, vp]),
        "lbm39_step": (i, [vp, i64]),
        "lbm39_sync": (i, [vp, i64, ctypes.POINTER(i64)]),
        "lbm39_read": (i, [vp, vp, vp, vp, vp]),
        "lbm39_read_host": (i, [vp, vp, vp, vp, vp]),
        "lbm39_stats": (i, [vp, ctypes.POINTER(lbm39_stats_t)]),
        "lbm39_checkpoint_bytes": (sz, [vp]),
        "lbm39_save": (i, [vp, vp]),
        "lbm39_load": (i, [vp, vp]),
        "lbm39_selftest_exp": (i, [vp, vp, vp, i64, vp]),
        "lbm39_selftest_rcp": (i, [vp, vp, vp, vp, vp, i64, vp]),
        "lbm39_selftest_dfma": (i, [ctypes.POINTER(ctypes.c_double), vp, sz, vp]),
        "lbm39_conserved_noalloc": (i, [vp, vp]),
        "lbm39_diag_fields": (i, [vp, vp, vp]),
        "lbm39_batch_query_bytes": (i, [ctypes.c_int32, i64, ctypes.POINTER(sz)]),
        "lbm39_batch_create": (i, [ctypes.c_int32, i64, ctypes.c_int32, ctypes.c_int32, vp, vp,
                                   ctypes.POINTER(vp)]),
        "lbm39_batch_set": (i, [vp, vp, vp, ctypes.c_int32]),
        "lbm39_batch_run": (i, [vp, i64]),
        "lbm39_batch_destroy": (None, [vp]),
        "lbm39_destroy": (None, [vp]),
        "lbm39_strerror": (ctypes.c_char_p, [i]),
        # lbm39_poly.h: the polynomial-equilibrium comparison model
        "lbm39_poly_query_bytes": (i, [P, ctypes.POINTER(sz), ctypes.POINTER(sz)]),
        "lbm39_poly_create": (i, [P, vp, vp, vp, ctypes.POINTER(vp)]),
        "lbm39_poly_init": (i, [vp, vp, vp, vp]),
        "lbm39_poly_step": (i, [vp, i64]),
        "lbm39_poly_read": (i, [vp, vp, vp, vp, vp]),
        "lbm39_poly_conserved": (i, [vp, vp]),
        "lbm39_poly_time": (i64, [vp]),
        "lbm39_poly_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def check(rc: int, where: str = "lbm39") -> None:
    if rc != LBM39_OK:
        raise LBM39Error(rc, where)


def lbm39_default_params(nx: int, ny: int, nz: int) -> lbm39_params:
    p = lbm39_params()
    _lib.lbm39_default_params(ctypes.byref(p), nx, ny, nz)
    return p


def lbm39_velocities(vel_ptr, w_ptr) -> int:
    return _lib.lbm39_velocities(vel_ptr, w_ptr)


def lbm39_query_bytes(p: lbm39_params):
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    rc = _lib.lbm39_query_bytes(ctypes.byref(p), ctypes.byref(a), ctypes.byref(b))
    return rc, a.value, b.value


def lbm39_create(p: lbm39_params, vel_ptr, w_ptr, pop_ptr, aux_ptr, mask_ptr, stream_ptr):
    """Returns (rc, handle)."""
    h = ctypes.c_void_p()
    rc = _lib.lbm39_create(ctypes.byref(p), vel_ptr, w_ptr, pop_ptr, aux_ptr, mask_ptr,
                           stream_ptr, ctypes.byref(h))
    return rc, h.value


def lbm39_init(h, rho, u, T) -> int:
    return _lib.lbm39_init(h, rho, u, T)


def lbm39_init_host(h, rho, u, T) -> int:
    return _lib.lbm39_init_host(h, rho, u, T)


def lbm39_step(h, nsteps: int) -> int:
    return _lib.lbm39_step(h, nsteps)


def lbm39_sync(h, timeout_us: int = -1):
    """Returns (rc, failed_cells)."""
    n = ctypes.c_int64()
    rc = _lib.lbm39_sync(h, timeout_us, ctypes.byref(n))
    return rc, n.value


def lbm39_read(h, rho, u, T, p) -> int:
    return _lib.lbm39_read(h, rho, u, T, p)


def lbm39_read_host(h, rho, u, T, p) -> int:
    return _lib.lbm39_read_host(h, rho, u, T, p)


def lbm39_stats(h):
    s = lbm39_stats_t()
    rc = _lib.lbm39_stats(h, ctypes.byref(s))
    return rc, s


def lbm39_checkpoint_bytes(h) -> int:
    return _lib.lbm39_checkpoint_bytes(h)


def lbm39_save(h, buf) -> int:
    return _lib.lbm39_save(h, buf)


def lbm39_load(h, buf) -> int:
    return _lib.lbm39_load(h, buf)


def lbm39_selftest_dfma(scratch, nbytes: int, stream):
    """Returns (rc, TFLOP/s)."""
    t = ctypes.c_double()
    rc = _lib.lbm39_selftest_dfma(ctypes.byref(t), scratch, nbytes, stream)
    return rc, t.value


def lbm39_selftest_exp(x, y, ref, n: int, stream) -> int:
    return _lib.lbm39_selftest_exp(x, y, ref, n, stream)


def lbm39_selftest_rcp(x, y, ref, y32, ref32, n: int, stream) -> int:
    return _lib.lbm39_selftest_rcp(x, y, ref, y32, ref32, n, stream)


def lbm39_diag_fields(h, eps, n_upd) -> int:
    return _lib.lbm39_diag_fields(h, eps, n_upd)


def lbm39_conserved_noalloc(h, sums5_host) -> int:
    return _lib.lbm39_conserved_noalloc(h, sums5_host)


def lbm39_batch_query_bytes(max_lattices: int, max_cells: int):
    b = ctypes.c_size_t()
    rc = _lib.lbm39_batch_query_bytes(max_lattices, max_cells, ctypes.byref(b))
    return rc, b.value


def lbm39_batch_create(max_lattices, max_cells, precision, graph_steps, buf, stream):
    """Returns (rc, handle)."""
    h = ctypes.c_void_p()
    rc = _lib.lbm39_batch_create(max_lattices, max_cells, precision, graph_steps, buf, stream,
                                 ctypes.byref(h))
    return rc, h.value


def lbm39_batch_set(b, handles, t_end) -> int:
    n = len(handles)
    arr = (ctypes.c_void_p * max(n, 1))(*handles)
    te = (ctypes.c_int64 * max(n, 1))(*[int(t) for t in t_end])
    return _lib.lbm39_batch_set(b, ctypes.cast(arr, ctypes.c_void_p),
                                ctypes.cast(te, ctypes.c_void_p), n)


def lbm39_batch_run(b, nsteps: int) -> int:
    return _lib.lbm39_batch_run(b, nsteps)


def lbm39_batch_destroy(b) -> None:
    _lib.lbm39_batch_destroy(b)


def lbm39_destroy(h) -> None:
    _lib.lbm39_destroy(h)


def lbm39_strerror(code: int) -> str:
    return _lib.lbm39_strerror(code).decode()


def exported_symbols() -> list:
    return [n for n in dir(_lib) if n.startswith("lbm39_")]


# --- lbm39_poly.h ---------------------------------------------------------------------------

def lbm39_poly_query_bytes(p: lbm39_params):
    a = ctypes.c_size_t()
    b = ctypes.c_size_t()
    rc = _lib.lbm39_poly_query_bytes(ctypes.byref(p), ctypes.byref(a), ctypes.byref(b))
    return rc, a.value, b.value


def lbm39_poly_create(p: lbm39_params, pop_ptr, aux_ptr, stream_ptr):
    """Returns (rc, handle)."""
    h = ctypes.c_void_p()
    rc = _lib.lbm39_poly_create(ctypes.byref(p), pop_ptr, aux_ptr, stream_ptr, ctypes.byref(h))
    return rc, h.value


def lbm39_poly_init(h, rho, u, T) -> int:
    return _lib.lbm39_poly_init(h, rho, u, T)


def lbm39_poly_step(h, nsteps: int) -> int:
    return _lib.lbm39_poly_step(h, nsteps)


def lbm39_poly_read(h, rho, u, T, p) -> int:
    return _lib.lbm39_poly_read(h, rho, u, T, p)


def lbm39_poly_conserved(h, sums5_host) -> int:
    return _lib.lbm39_poly_conserved(h, sums5_host)


def lbm39_poly_time(h) -> int:
    return _lib.lbm39_poly_time(h)


def lbm39_poly_destroy(h) -> None:
    _lib.lbm39_poly_destroy(h)
