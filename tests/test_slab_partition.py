"""Domain decomposition of the step on CPU: two gloo ranks each advance one z-slab of a
periodic box, exchanging three halo layers per step, and together reproduce the unsplit run
bit for bit.

The step is local except for streaming over shifts of up to 3 cells (Sec. 3), so a slab that
carries 3 extra layers on each side, refreshed every step with the neighbour's pre-collision
state (f, g and the multipliers of the warm start), collides its own cells exactly as the
whole lattice would and pulls streamed values only from cells it holds correctly.  The halo
cells themselves pull from beyond the slab and are overwritten at the next exchange.  This is
the exchange a multi-GPU build would make (3 layers x 78 populations + 13 multipliers per face
cell); runs here have one GPU, so it is verified with the oracle."""
import os
import socket
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
H = 3  # halo layers: the longest lattice shift
SHAPE = (8, 10, 12)  # (nz, ny, nx)
STEPS = 12


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _setup():
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from gpu_helpers import oracle_cfg
    from oracle import oracle39 as o
    from paper_1910_13515_gb300 import inputs
    s = inputs.box(seed=3, shape=SHAPE)
    return o, s, oracle_cfg(s)


def _layers(a, z0, z1, nz, plane):
    """Rows of the cells with z in [z0, z1) (wrapped), as (z1 - z0) * plane rows."""
    return np.concatenate([a[(z % nz) * plane:(z % nz + 1) * plane] for z in range(z0, z1)])


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    o, s, cfg = _setup()
    nz, ny, nx = SHAPE
    plane = nx * ny
    full = o.init(cfg, s.mask, s.rho, s.u, s.T)
    nzl = nz // world
    z0, z1 = rank * nzl, (rank + 1) * nzl
    ext = o.Config(**{**cfg.__dict__, "nz": nzl + 2 * H})
    st = o.State(ext, _layers(full.mask.reshape(-1, 1), z0 - H, z1 + H, nz, plane).ravel(),
                 _layers(full.f, z0 - H, z1 + H, nz, plane),
                 _layers(full.g, z0 - H, z1 + H, nz, plane),
                 _layers(full.lam, z0 - H, z1 + H, nz, plane),
                 on_fb=_layers(full.on_fb, z0 - H, z1 + H, nz, plane))
    lo, hi = (rank - 1) % world, (rank + 1) % world
    n_halo = H * plane
    for _ in range(STEPS):
        # pre-collision state of the interior layers next to each face -> the neighbours
        send_lo = [torch.from_numpy(np.ascontiguousarray(a[n_halo:2 * n_halo]))
                   for a in (st.f, st.g, st.lam, st.on_fb)]
        send_hi = [torch.from_numpy(np.ascontiguousarray(a[-2 * n_halo:-n_halo]))
                   for a in (st.f, st.g, st.lam, st.on_fb)]
        recv_lo = [torch.empty_like(t) for t in send_lo]
        recv_hi = [torch.empty_like(t) for t in send_hi]
        reqs = []
        for t in send_lo:
            reqs.append(dist.isend(t, lo, tag=1))
        for t in send_hi:
            reqs.append(dist.isend(t, hi, tag=2))
        for t in recv_hi:   # the upper neighbour's lowest interior layers
            reqs.append(dist.irecv(t, hi, tag=1))
        for t in recv_lo:   # the lower neighbour's highest interior layers
            reqs.append(dist.irecv(t, lo, tag=2))
        for r in reqs:
            r.wait()
        for a, t in zip((st.f, st.g, st.lam, st.on_fb), recv_lo):
            a[:n_halo] = t.numpy()
        for a, t in zip((st.f, st.g, st.lam, st.on_fb), recv_hi):
            a[-n_halo:] = t.numpy()
        assert o.step(st, 1) == 0
    out[rank] = (st.f[n_halo:-n_halo].copy(), st.g[n_halo:-n_halo].copy(),
                 st.lam[n_halo:-n_halo].copy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_slabs_with_halo_exchange_equal_the_unsplit_run():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn")
    o, s, cfg = _setup()
    st = o.init(cfg, s.mask, s.rho, s.u, s.T)
    assert o.step(st, STEPS) == 0
    f = np.concatenate([out[r][0] for r in range(world)])
    g = np.concatenate([out[r][1] for r in range(world)])
    lam = np.concatenate([out[r][2] for r in range(world)])
    assert np.array_equal(f, st.f) and np.array_equal(g, st.g) and np.array_equal(lam, st.lam)
