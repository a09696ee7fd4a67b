"""Pins of the oracle's exact-rational Hermite stencils (Sec. 3.2)."""
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import coeffs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "stencils_eq3_8_3_10_3_18.txt")


def _golden():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        rows.append((f[0], int(f[1]), f[2:]))
    return rows


@pytest.mark.parametrize("name,nd,printed", _golden())
def test_printed_face_coefficients(name, nd, printed):
    """Every coefficient printed in Eq. 3.8, 3.10 and 3.18 is reproduced exactly."""
    got = coeffs.eval_functional(coeffs.stencil_poly(name), Fr(1, 2), nd)
    for k, p in enumerate(printed):
        if p == "omitted":
            continue
        assert got[k] == Fr(p), (name, nd, k, got[k], p)


def test_r7_value_term_omitted_in_print():
    """Eq. 3.18 prints the r7 face value without its Qbar_{i-1} term; the
    conditions force -223/1260, which makes the coefficients sum to 1."""
    got = coeffs.eval_functional(coeffs.stencil_poly("r7"), Fr(1, 2), 0)
    assert got[1] == Fr(-223, 1260)
    assert sum(got[:5]) == 1


@pytest.mark.parametrize("name", list(coeffs.STENCILS))
def test_polynomial_reproduction(name):
    """Brute force: data sampled from any polynomial of the stencil's degree is
    reproduced exactly (cell averages and slope averages in, values out)."""
    avgs, slopes = coeffs.STENCILS[name]
    deg = len(avgs) + len(slopes) - 1
    C = coeffs.stencil_poly(name)
    rng = np.random.default_rng(1)
    for _ in range(3):
        a = [Fr(int(x), 7) for x in rng.integers(-9, 10, deg + 1)]
        P = lambda x: sum(c * x ** n for n, c in enumerate(a))
        Pint = lambda lo, hi: sum(c * (hi ** (n + 1) - lo ** (n + 1)) / (n + 1) for n, c in enumerate(a))
        d = [Fr(0)] * 10
        for k in range(-2, 3):
            lo, hi = Fr(2 * k - 1, 2), Fr(2 * k + 1, 2)
            d[k + 2] = Pint(lo, hi)
            d[5 + k + 2] = P(hi) - P(lo)
        for xi in (Fr(1, 2), Fr(-1, 2), Fr(1, 3)):
            val = sum(r * x for r, x in zip(coeffs.eval_functional(C, xi, 0), d))
            assert val == P(xi)


def test_gauss_legendre_weights():
    for m in (2, 3, 4):
        x, w = coeffs.gauss_legendre_unit(m)
        assert abs(w.sum() - 1) < 1e-15
        for k in range(2 * m):
            exact = 0.0 if k % 2 else 2 * 0.5 ** (k + 1) / (k + 1)
            assert abs((w * x ** k).sum() - exact) < 1e-15
