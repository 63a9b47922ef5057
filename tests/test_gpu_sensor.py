"""The Knudsen sensor's branch decision (Eq. DeltaAvg, Eq. alpha) on the GPU at values of
39 eps placed just below and above each threshold.

Each cell's f is the equilibrium of a uniform state perturbed in the null space of the
conserved moments (mass, momentum and sum f|xi|^2, with g at equilibrium), so rho, u and T,
the targets and the multipliers are those of the unperturbed state, and 39 eps equals
sum_i |delta_i| exactly as designed.  Values from 1e-3 down to 1e-7 away from 0.39, 3.9 and
39 cover both the FP32 screen and its FP64 fallback.  One step on the GPU must match the
oracle to parity (a wrong branch changes 1/tau_eff by 5-35% in that cell) and give the same
histogram of branches."""
import numpy as np
import pytest
import torch

from gpu_helpers import TOL, lib_to_oracle_perm, oracle_cfg, rel_diffs
from oracle import oracle39 as o
from paper_1910_13515_gb300 import inputs

pytestmark = pytest.mark.gpu

OFFSETS = [-1e-3, -1e-4, -2e-5, -5e-6, -1e-7, 1e-7, 5e-6, 2e-5, 1e-4, 1e-3]


def designed_sums(n):
    vals = [t + d for t in (0.39, 3.9, 39.0) for d in OFFSETS]
    rng = np.random.default_rng(5)
    vals += list(rng.uniform(0.0, 60.0, n - len(vals)))
    return np.array(vals[:n])


def null_perturbation(feq, xi, s39, rng):
    """delta (oracle order) with sum_i delta_i feq_i phi(xi_i) = 0 for phi in {1, xi, |xi|^2}
    and sum_i |delta_i| = s39."""
    A = np.stack([feq, feq * xi[:, 0], feq * xi[:, 1], feq * xi[:, 2], feq * (xi ** 2).sum(1)])
    _, _, vt = np.linalg.svd(A)
    basis = vt[A.shape[0]:].T  # 39 x 34, orthonormal null space
    d = basis @ rng.standard_normal(basis.shape[1])
    return d * (s39 / np.abs(d).sum())


def test_alpha_branch_decisions_near_thresholds():
    from paper_1910_13515_gb300 import build
    build.build()
    from paper_1910_13515_gb300.lattice import Lattice
    s = inputs.uniform(4, 4, 4, u=(0.3, -0.1, 0.2), T=0.5, tau=0.6)
    N = s.ncells
    L = Lattice.from_setup(s)
    st = o.init(oracle_cfg(s), s.mask, s.rho, s.u, s.T)
    xi, _, _ = o.lattice()
    xi = np.asarray(xi, np.float64)
    sums = designed_sums(N)
    rng = np.random.default_rng(9)
    perm = lib_to_oracle_perm()  # perm[j] = library index of oracle velocity j
    buf = L.checkpoint()
    Np = (N + 63) // 64 * 64
    pops = buf[256:].view(torch.float64)[:78 * Np].view(78, Np)
    f_lib = pops[:39, :N].cpu().numpy().copy()
    for c in range(N):
        d = null_perturbation(st.f[c], xi, sums[c], rng)
        st.f[c] = st.f[c] * (1.0 + d)
        f_lib[perm, c] = f_lib[perm, c] * (1.0 + d)
    pops[:39, :N] = torch.as_tensor(f_lib, device=buf.device)
    L.restore(buf)
    L.step(1)
    assert L.sync() == 0
    assert o.step(st, 1) == 0
    assert list(L.stats().eps_hist) == list(st.stats.eps_hist)
    d = rel_diffs(L.read_numpy(), o.macros(st), s.mask, s.gamma)
    assert max(d) <= TOL, d
    # the designed sums did land on both sides of every threshold
    assert all(h > 0 for h in st.stats.eps_hist)
