"""Shared helpers of the GPU parity tests: run a setup on both sides, compare fields."""
import numpy as np
import torch

from oracle import oracle39 as o

TOL = 1e-11  # max relative difference in rho/u/T vs the FP64 oracle (FP64 path)


def oracle_cfg(s, **kw):
    return o.Config(nx=s.nx, ny=s.ny, nz=s.nz, periodic=s.periodic, gamma=s.gamma, tau=s.tau,
                    kn_sensor=s.kn_sensor, rho_inf=s.rho_inf, u_inf=s.u_inf, T_inf=s.T_inf, **kw)


def run_oracle(s, nsteps, **kw):
    st = o.init(oracle_cfg(s, **kw), s.mask, s.rho, s.u, s.T)
    failed = o.step(st, nsteps)
    return st, failed


def rel_diffs(a, b, mask, gamma):
    """(rho, u, T) relative differences over fluid cells; u relative to max(|u|, c_s)."""
    ra, ua, Ta = a[:3]
    rb, ub, Tb = b[:3]
    fl = mask == 0
    dr = np.abs(ra[fl] - rb[fl]).max() / np.abs(rb[fl]).max()
    cs = np.sqrt(gamma * np.abs(Tb[fl]).max())
    du = np.abs(ua[:, fl] - ub[:, fl]).max() / max(np.abs(ub[:, fl]).max(), cs)
    dT = np.abs(Ta[fl] - Tb[fl]).max() / np.abs(Tb[fl]).max()
    return dr, du, dT


def lib_to_oracle_perm():
    """perm[j] = library index of oracle velocity j."""
    from paper_1910_13515_gb300.lattice import velocities
    lv, _ = velocities()
    ov, _, _ = o.lattice()
    idx = {tuple(v): i for i, v in enumerate(lv)}
    return np.array([idx[tuple(v)] for v in ov])


def fallback_flags(lam):
    """The oracle's per-cell "on the fallback" flags of multipliers (n, 13) read from the
    library's state: the library marks a cell on the fallback by lambda_9 = -0 inside the
    embedding of the five fallback multipliers (lambda_4 = lambda_5 = lambda_6, the other
    second- and third-order multipliers +0)."""
    lam = np.asarray(lam)
    rest = np.delete(lam[:, 7:], 2, axis=1)
    bits = rest.view(np.uint64)
    return ((lam[:, 9] == 0) & np.signbit(lam[:, 9]) & (bits == 0).all(axis=1)
            & (lam[:, 4].view(np.uint64) == lam[:, 5].view(np.uint64))
            & (lam[:, 5].view(np.uint64) == lam[:, 6].view(np.uint64))).astype(np.uint8)


def patch_from_checkpoint(L, buf, cx, cy, cz, r=3):
    """Populations (oracle order) and multipliers of the (2r+1)^d patch around (cx,cy,cz) from a
    checkpoint taken at even time (pre-collision populations in their own slots)."""
    p = L.params
    nx, ny, nz = p.nx, p.ny, p.nz
    N = nx * ny * nz
    Np = (N + 63) // 64 * 64
    body = buf[256:].view(torch.float64)
    pops = body[: 78 * Np].view(78, Np)
    lams = body[78 * Np: 78 * Np + 13 * Np].view(13, Np)  # multipliers lead the solver state
    rz = r if nz > 1 else 0
    xs = [(cx + d) % nx for d in range(-r, r + 1)]
    ys = [(cy + d) % ny for d in range(-r, r + 1)]
    zs = [(cz + d) % nz for d in range(-rz, rz + 1)]
    cells = np.array([x + nx * (y + ny * z) for z in zs for y in ys for x in xs])
    ci = torch.as_tensor(cells, device=buf.device)
    P = pops[:, ci].cpu().numpy()   # (78, n)
    lam = lams[:, ci].cpu().numpy()  # (13, n)
    perm = lib_to_oracle_perm()
    f = P[:39][perm].T.copy()
    g = P[39:][perm].T.copy()
    return cells, f, g, lam.T.copy(), (len(xs), len(ys), len(zs))
