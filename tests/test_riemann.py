"""Self-checks of the exact Riemann solver used as the Sod pin: the textbook star state of
Sod's problem and the Rankine-Hugoniot / isentropic relations across its waves."""
import math

import numpy as np

from oracle import riemann


def test_classic_sod_star_state():
    ps, us = riemann.star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    assert abs(ps - 0.30313) < 1e-5 and abs(us - 0.92745) < 1e-5
    assert abs(riemann.shock_speed(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4) - 1.7522) < 1e-4


def test_rankine_hugoniot_across_the_shock():
    g = 1.4
    for (rl, pl, rr, pr) in [(1, 1, 0.125, 0.1), (0.7, 0.6, 0.2, 0.05), (1, 0.5, 0.125, 0.05)]:
        ps, us = riemann.star_state(rl, 0, pl, rr, 0, pr, g)
        S = riemann.shock_speed(rl, 0, pl, rr, 0, pr, g)
        r, u, p = riemann.sample(np.array([S - 1e-9, S + 1e-9]), rl, 0, pl, rr, 0, pr, g)
        E = p / (g - 1) + 0.5 * r * u * u
        # mass, momentum and energy fluxes in the shock frame are continuous
        m = r * (u - S)
        mom = r * u * (u - S) + p
        en = (E + p) * u - S * E
        assert abs(m[0] - m[1]) < 1e-10 and abs(mom[0] - mom[1]) < 1e-10
        assert abs(en[0] - en[1]) < 1e-10


def test_rarefaction_is_isentropic_and_continuous():
    g = 1.4
    rl, pl, rr, pr = 1.0, 1.0, 0.125, 0.1
    ps, us = riemann.star_state(rl, 0, pl, rr, 0, pr, g)
    al = math.sqrt(g * pl / rl)
    xi = np.linspace(-al, us - al * (ps / pl) ** ((g - 1) / (2 * g)), 50)
    r, u, p = riemann.sample(xi, rl, 0, pl, rr, 0, pr, g)
    assert np.allclose(p / r**g, pl / rl**g, rtol=1e-12)          # entropy constant
    a = np.sqrt(g * p / r)
    assert np.allclose(u + 2 * a / (g - 1), 2 * al / (g - 1), rtol=1e-12)  # J+ invariant
    assert np.allclose(u - a, xi, atol=1e-12)                     # characteristic fan


def test_symmetric_problem():
    r, u, p = riemann.sample(np.array([-0.3, 0.3]), 1, 0.5, 1, 1, -0.5, 1, 1.4)
    assert abs(u[0]) < 1e-12 and abs(u[1]) < 1e-12 and abs(r[0] - r[1]) < 1e-12
