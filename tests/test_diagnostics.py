"""Host diagnostics: surface cells and the pressure coefficient of the NACA0012 setup, against
brute force and fields with a known C_p."""
import numpy as np

from paper_1910_13515_gb300 import diagnostics, inputs


def small_naca():
    return inputs.naca(nx=256, ny=128, chord=50)


def test_surface_cells_brute_force():
    s = small_naca()
    m = s.mask.reshape(s.ny, s.nx)
    want = []
    for y in range(s.ny):
        for x in range(s.nx):
            if m[y, x] != inputs.M_FLUID:
                continue
            nb = [(x - 1, y), (x + 1, y), (x, y - 1), (x, y + 1)]
            if any(0 <= a < s.nx and 0 <= b < s.ny and m[b, a] == inputs.M_SOLID for a, b in nb):
                want.append(y * s.nx + x)
    got = diagnostics.surface_cells(s)
    assert len(want) > 50 and list(got) == want


def test_surface_is_mirror_symmetric_at_zero_incidence():
    s = small_naca()
    xu, _, xl, _ = diagnostics.surface_cp(s, np.ones(s.ncells), np.full(s.ncells, s.T_inf))
    np.testing.assert_array_equal(xu, xl)
    assert xu.min() < 0.05 and xu.max() > 0.9  # the last cells of the thin trailing edge are fluid


def test_cp_of_known_pressure_fields():
    s = small_naca()
    q = 0.5 * s.rho_inf * s.u_inf[0] ** 2
    rho = np.full(s.ncells, s.rho_inf)
    _, cu, _, cl = diagnostics.surface_cp(s, rho, np.full(s.ncells, s.T_inf))
    assert np.abs(cu).max() == 0 and np.abs(cl).max() == 0
    # p = p_inf + q everywhere -> C_p = 1; p = p_inf - q/2 with T fixed -> C_p = -1/2
    _, cu, _, cl = diagnostics.surface_cp(s, rho, np.full(s.ncells, s.T_inf + q / s.rho_inf))
    np.testing.assert_allclose(np.concatenate([cu, cl]), 1.0, rtol=1e-13)
    rho2 = np.full(s.ncells, s.rho_inf - 0.5 * q / s.T_inf)
    _, cu, _, cl = diagnostics.surface_cp(s, rho2, np.full(s.ncells, s.T_inf))
    np.testing.assert_allclose(np.concatenate([cu, cl]), -0.5, rtol=1e-13)
    # p growing linearly along x: C_p follows x/C
    cells = np.arange(s.ncells)
    xc = ((cells % s.nx) - s.extra["x_le"]) / s.extra["chord"]
    T = s.T_inf + q * xc / s.rho_inf
    xu, cu, xl, cl = diagnostics.surface_cp(s, rho, T)
    np.testing.assert_allclose(cu, xu, atol=1e-13)
    np.testing.assert_allclose(cl, xl, atol=1e-13)
