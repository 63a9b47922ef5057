"""The precision form's storage representation, emulated on the FP64 oracle.

The precision form keeps every population as the FP32 rounding of its deviation from a
reference population.  Emulating that rounding after each oracle step shows what the
representation alone costs, independent of the GPU: on the Ma 1.5 airfoil the rest
reference (the equilibrium at rho = 1, u = 0, T = 0.5) stores the populations that point
against the flow four to five orders of magnitude below their references, i.e. on a grid of
~1e-3 of themselves, while the far-field reference stores the undisturbed flow exactly.  The
storage noise of the rest reference also forces Newton updates that FP64 storage does not
need; with the far-field reference the solve takes the FP64 counts."""
import numpy as np

from paper_1910_13515_gb300 import inputs


def _airfoil(oracle):
    s = inputs.naca(nx=96, ny=48, chord=24, x_le=24)
    cfg = oracle.Config(nx=s.nx, ny=s.ny, nz=s.nz, periodic=s.periodic, gamma=s.gamma,
                        tau=s.tau, kn_sensor=s.kn_sensor, rho_inf=s.rho_inf, u_inf=s.u_inf,
                        T_inf=s.T_inf)
    return s, cfg


def _l1(a, b, fl):
    (ra, ua, Ta), (rb, ub, Tb) = a[:3], b[:3]
    return max(np.abs(ra[fl] - rb[fl]).mean() / np.abs(rb[fl]).mean(),
               np.abs(ua[:, fl] - ub[:, fl]).mean() / np.sqrt((ub[:, fl] ** 2).sum(0)).mean(),
               np.abs(Ta[fl] - Tb[fl]).mean() / np.abs(Tb[fl]).mean())


def _run(oracle, s, cfg, nsteps, ref):
    """nsteps oracle steps; after each, populations rounded to FP32 deviations from the
    equilibrium of the reference state `ref` (None: FP64 storage).  Returns (state, Newton
    updates per step)."""
    st = oracle.init(cfg, s.mask, s.rho, s.u, s.T)
    if ref is not None:
        feq, geq, _, status = oracle.equilibrium(cfg, *ref)
        assert status == 0
    upd = []
    for _ in range(nsteps):
        u0 = st.stats.newton_updates
        oracle.step(st, 1)
        upd.append(st.stats.newton_updates - u0)
        if ref is not None:
            st.f[:] = feq + (st.f - feq).astype(np.float32).astype(np.float64)
            st.g[:] = geq + (st.g - geq).astype(np.float32).astype(np.float64)
    return st, upd


def test_far_field_reference_stores_the_airfoil_flow_finely(oracle):
    s, cfg = _airfoil(oracle)
    fl = s.mask == 0
    n = 20
    exact, up64 = _run(oracle, s, cfg, n, None)
    rest, up_rest = _run(oracle, s, cfg, n, (1.0, np.zeros(3), 0.5))
    far, up_far = _run(oracle, s, cfg, n, (s.rho_inf, np.array(s.u_inf), s.T_inf))
    e_rest = _l1(oracle.macros(rest), oracle.macros(exact), fl)
    e_far = _l1(oracle.macros(far), oracle.macros(exact), fl)
    assert e_far < 1e-7 < 1e-5 < e_rest, (e_far, e_rest)
    # storage noise: in the first steps, while most of the lattice is undisturbed, the rest
    # reference forces updates there; the far field takes the FP64 counts throughout
    assert sum(up_rest[:6]) > 1.5 * sum(up64[:6]), (up_rest[:6], up64[:6])
    assert abs(sum(up_far) - sum(up64)) <= 0.01 * sum(up64), (sum(up_far), sum(up64))
