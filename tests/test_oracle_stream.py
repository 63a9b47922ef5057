"""Brute-force pins of the oracle's streaming with masks (Sec. 3 collide-and-stream and the
boundary conditions of Sec. 4 of arXiv:1910.13515), with unique tagged values per (cell, i)."""
import itertools

import numpy as np
import pytest

from paper_1910_13515_gb300 import inputs


def tagged(N):
    f = (np.arange(N)[:, None] * 100 + np.arange(39)[None, :]).astype(float) + 0.25
    g = -f
    return f, g


def brute(oracle, nx, ny, nz, mask, fpost, feq_inf):
    """Direct index arithmetic: h_i(x) = h*_i(x - xi_i) (periodic wrap); solid source ->
    h*_opp(i)(x); freestream source -> h^eq_inf; outflow source -> the cell with x clamped into
    [3, nx-4] (or h^eq_inf if that cell is freestream)."""
    vel, _, opp = oracle.lattice()
    out = np.zeros_like(fpost)
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        c = x + nx * (y + ny * z)
        if mask[c] != 0:
            continue
        for i in range(39):
            sx, sy, sz = (x - vel[i, 0]) % nx, (y - vel[i, 1]) % ny, (z - vel[i, 2]) % nz
            s = sx + nx * (sy + ny * sz)
            if mask[s] == 1:
                out[c, i] = fpost[c, opp[i]]
            elif mask[s] == 0:
                out[c, i] = fpost[s, i]
            elif mask[s] == 2:
                out[c, i] = feq_inf[i]
            else:
                xc = min(max(sx, 3), nx - 4)
                cc = xc + nx * (sy + ny * sz)
                out[c, i] = feq_inf[i] if mask[cc] == 2 else fpost[cc, i]
    return out


@pytest.mark.parametrize("dims", [(5, 4, 3), (7, 1, 1), (2, 2, 2), (1, 1, 1), (4, 1, 3)])
def test_periodic_streaming_brute_force(oracle, dims):
    nx, ny, nz = dims
    N = nx * ny * nz
    cfg = oracle.Config(nx=nx, ny=ny, nz=nz)
    mask = np.zeros(N, np.uint8)
    f, g = tagged(N)
    fo, go = oracle.stream(cfg, mask, f, g, np.zeros(39), np.zeros(39))
    assert np.array_equal(fo, brute(oracle, nx, ny, nz, mask, f, np.zeros(39)))
    assert np.array_equal(go, -fo)
    # a permutation of the post-collision values: mass conserved exactly
    assert np.array_equal(np.sort(fo.ravel()), np.sort(f.ravel()))


def test_bounce_back_brute_force(oracle):
    nx, ny, nz = 9, 8, 7
    N = nx * ny * nz
    rng = np.random.default_rng(5)
    mask = np.zeros(N, np.uint8)
    mask[rng.choice(N, 25, replace=False)] = 1
    mask[4 + nx * (4 + ny * 3)] = 1
    cfg = oracle.Config(nx=nx, ny=ny, nz=nz)
    f, g = tagged(N)
    fo, go = oracle.stream(cfg, mask, f, g, np.zeros(39), np.zeros(39))
    assert np.array_equal(fo, brute(oracle, nx, ny, nz, mask, f, np.zeros(39)))
    fl = mask == 0
    # every fluid post value lands exactly once in a fluid cell
    assert np.array_equal(np.sort(fo[fl].ravel()), np.sort(f[fl].ravel()))


def test_freestream_and_outflow_cells_brute_force(oracle):
    st = inputs.naca(nx=40, ny=24, chord=10, x_le=12)
    N = st.ncells
    cfg = oracle.Config(nx=st.nx, ny=st.ny, nz=1, periodic=st.periodic)
    f, g = tagged(N)
    feq_inf = np.arange(39) + 0.5
    fo, go = oracle.stream(cfg, st.mask, f, g, feq_inf, -feq_inf)
    assert np.array_equal(fo, brute(oracle, st.nx, st.ny, 1, st.mask, f, feq_inf))
    assert (st.mask == 1).sum() > 5 and (st.mask == 3).sum() > 0


def test_riemann_tube_outflow_both_ends(oracle):
    st = inputs.sod(nx=16)
    cfg = oracle.Config(nx=16, periodic=st.periodic)
    f, g = tagged(16)
    fo, go = oracle.stream(cfg, st.mask, f, g, np.full(39, 7.0), np.full(39, -7.0))
    assert np.array_equal(fo, brute(oracle, 16, 1, 1, st.mask, f, np.full(39, 7.0)))
