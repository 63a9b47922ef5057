"""The CUDA path's polynomial equilibrium (csrc/poly_eq.cuh: the scalar quartic in xi.u with
per-shell coefficients), compiled for the host, against the oracle's tensor-Hermite form:
checks the hand-contracted coefficients without a GPU.  Needs nvcc, not a GPU."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def host_lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("polyhost") / "polyhost.so")
    subprocess.check_call([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O2", "-Xcompiler",
                           "-fPIC", "-shared", "-gencode", "arch=compute_103a,code=sm_103a",
                           "-o", out, os.path.join(ROOT, "tests", "poly_eq_host.cu")])
    return ctypes.CDLL(out)


@pytest.fixture(scope="module")
def poly():
    from oracle import oracle39, poly39
    oracle39.build()
    return poly39


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


@pytest.mark.parametrize("umax,Trange,tol", [(0.3, (0.55, 0.8), 2e-14),
                                             (0.8, (0.3, 1.2), 2e-13)])
def test_scalar_form_equals_tensor_form(host_lib, poly, umax, Trange, tol):
    lv = np.zeros((39, 3), np.int32)
    host_lib.poly_velocities_host(_p(lv))
    vel, w = poly.lattice()
    perm = [int(np.where((vel == lv[i]).all(axis=1))[0][0]) for i in range(39)]
    rng = np.random.default_rng(11)
    n = 3000
    rho = rng.uniform(0.5, 2.0, n)
    u = np.ascontiguousarray(rng.uniform(-umax, umax, (3, n)))
    T = rng.uniform(*Trange, n)
    out = np.zeros((n, 39))
    host_lib.poly_feq_host(_p(rho), _p(u), _p(T), ctypes.c_longlong(n), _p(out))
    ref = poly.feq(rho, u.T, T)[:, perm]
    err = np.abs(out - ref) / (rho[:, None] * w[perm][None, :])
    assert err.max() < tol, err.max()
