"""Pins of the oracle's D3Q39 lattice (Sec. 3 of arXiv:1910.13515)."""
import itertools
import os

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _shells():
    rows = []
    for line in open(os.path.join(GOLDEN, "d3q39_shells.txt")):
        if line.startswith("#") or not line.strip():
            continue
        a, b, c, cnt, c2 = map(int, line.split())
        rows.append(((a, b, c), cnt, c2))
    return rows


def test_velocity_set_matches_paper_shells(oracle):
    vel, w, opp = oracle.lattice()
    assert vel.shape == (39, 3)
    assert len({tuple(v) for v in vel}) == 39
    for rep, cnt, c2 in _shells():
        orbit = set()
        for perm in itertools.permutations(rep):
            for signs in itertools.product((1, -1), repeat=3):
                orbit.add(tuple(s * p for s, p in zip(signs, perm)))
        assert len(orbit) == cnt
        for v in orbit:
            assert v in {tuple(x) for x in vel}
            assert sum(x * x for x in v) == c2
    assert sum(cnt for _, cnt, _ in _shells()) == 39


def test_opposites_and_symmetry(oracle):
    vel, w, opp = oracle.lattice()
    for i in range(39):
        assert np.array_equal(vel[opp[i]], -vel[i])
    s = {tuple(v) for v in vel}
    for v in vel:
        for perm in itertools.permutations(range(3)):
            assert tuple(v[list(perm)]) in s


def test_weights_are_a_degree7_gaussian_quadrature(oracle):
    """Shan's E^39_{3,7} weights integrate every monomial of degree <= 7 exactly against a
    Gaussian of variance c_s^2 = 2/3 (odd moments vanish; even ones are Gaussian moments)."""
    vel, w, _ = oracle.lattice()
    s2 = 2.0 / 3.0
    dfact = {0: 1, 2: 1, 4: 3, 6: 15}
    for p in range(8):
        for q in range(8 - p):
            for r in range(8 - p - q):
                mom = float((w * vel[:, 0] ** p * vel[:, 1] ** q * vel[:, 2] ** r).sum())
                if p % 2 or q % 2 or r % 2:
                    exact = 0.0
                else:
                    exact = dfact[p] * dfact[q] * dfact[r] * s2 ** ((p + q + r) // 2)
                assert abs(mom - exact) < 1e-13, (p, q, r, mom, exact)
    # the degree-8 moment xi_x^8 is NOT exact (a 7th-order set): 105 s2^4 vs lattice
    m8 = float((w * vel[:, 0] ** 8).sum())
    assert abs(m8 - 105 * s2**4) > 1e-3


def test_basis_monomials(oracle):
    for xi in [(1, 2, 3), (-3, 0, 2), (0, 0, 0)]:
        x, y, z = xi
        s = x * x + y * y + z * z
        ref = [1, x, y, z, x * x, y * y, z * z, x * y, x * z, y * z, x * s, y * s, z * s]
        assert np.array_equal(oracle.basis(xi), np.array(ref, float))


def test_alpha_table_golden(oracle):
    tau = 0.57
    for line in open(os.path.join(GOLDEN, "alpha_table.txt")):
        if line.startswith("#") or not line.strip():
            continue
        lo, hi, a = line.split()
        lo, hi = float(lo), float(hi)
        want = 1.0 / tau if a == "inv_tau" else float(a)
        assert oracle.alpha(lo, tau) == want
        inner = lo * 1.0000001 if lo > 0 else 1e-9
        assert oracle.alpha(inner, tau) == want
        if np.isfinite(hi):
            assert oracle.alpha(np.nextafter(hi, 0), tau) == want
            assert oracle.alpha(hi, tau) != want
