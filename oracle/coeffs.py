"""Exact-rational Hermite stencils of the ASE-DFF reconstruction (oracle side).

TEST INFRASTRUCTURE ONLY.  This module belongs to the FP64 CPU oracle; only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
leg of ``bench.py`` may import it.  The CUDA path derives its own tables.

Every stencil is a polynomial p(xi) on the local coordinate xi = (x - x_i)/dx
(cell i is xi in [-1/2, 1/2], cell i+k is [k-1/2, k+1/2]).  Its conditions
are the ones the paper states:

* cell averages   int_{I_{i+k}} p dxi            = Qbar_{i+k}
* slope averages  p(k+1/2) - p(k-1/2)            = dx * (Qbar_x)_{i+k}

  (the average over I_{i+k} of dp/dx, written in xi units).

Stencils (paper Sec. 3.2):

* ``S0``  {Qbar_{i-1}, Qbar_i, Qx_{i-1}}                    Eq. 3.7, degree 2
* ``S1``  {Qbar_i, Qbar_{i+1}, Qx_{i+1}}                    Eq. 3.7, degree 2
* ``S2``  {Qbar_{i-1}, Qbar_i, Qbar_{i+1}}                  Eq. 3.7, degree 2
* ``r5``  {Qbar_{i-1..i+1}, Qx_{i-1}, Qx_{i+1}}             Eq. 3.9-3.10, degree 4
* ``r7``  {Qbar_{i-2..i+2}, Qx_{i-1}, Qx_{i+1}}             Eq. 3.18, degree 6
* ``r9``  {Qbar_{i-2..i+2}, Qx_{i-2}, Qx_{i-1}, Qx_{i+1}, Qx_{i+2}}  Eq. 3.18, degree 8

Reading: the own-cell slope (Qx)_i is not a condition of any stencil.  With it
the printed coefficients of Eq. 3.8, 3.10 and 3.18 cannot be reproduced;
without it every printed coefficient is reproduced (Eq. 3.18's r7 value
formula drops the -223/1260 Qbar_{i-1} term that the conditions force).

The data vector used everywhere is
``d = [Qbar_{i-2}, ..., Qbar_{i+2}, dx*Qx_{i-2}, ..., dx*Qx_{i+2}]`` (10 entries).
"""
from fractions import Fraction as Fr

import numpy as np

NDATA = 10
# offsets of the cells whose averages / slopes enter each stencil
STENCILS = {
    "S0": ((-1, 0), (-1,)),
    "S1": ((0, 1), (1,)),
    "S2": ((-1, 0, 1), ()),
    "r5": ((-1, 0, 1), (-1, 1)),
    "r7": ((-2, -1, 0, 1, 2), (-1, 1)),
    "r9": ((-2, -1, 0, 1, 2), (-2, -1, 1, 2)),
}


def _avg_row(k, deg):
    """Row of the cell-average condition over [k-1/2, k+1/2] for xi^0..xi^deg."""
    a, b = Fr(2 * k - 1, 2), Fr(2 * k + 1, 2)
    return [(b ** (n + 1) - a ** (n + 1)) / (n + 1) for n in range(deg + 1)]


def _slope_row(k, deg):
    """Row of the slope-average condition p(k+1/2) - p(k-1/2)."""
    a, b = Fr(2 * k - 1, 2), Fr(2 * k + 1, 2)
    return [b ** n - a ** n for n in range(deg + 1)]


def _solve(A, B):
    """Exact Gauss-Jordan elimination: returns X with A X = B (lists of Fractions)."""
    n = len(A)
    M = [list(A[r]) + list(B[r]) for r in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        piv = M[c][c]
        M[c] = [x / piv for x in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [row[n:] for row in M]


def stencil_poly(name):
    """Exact polynomial-coefficient matrix C (deg+1 x 10) of a stencil.

    p(xi) = sum_n xi^n * sum_d C[n][d] * d[d]  reproduces the stencil's
    conditions for any data vector d.
    """
    avgs, slopes = STENCILS[name]
    deg = len(avgs) + len(slopes) - 1
    rows, rhs = [], []
    for k in avgs:
        rows.append(_avg_row(k, deg))
        e = [Fr(0)] * NDATA
        e[k + 2] = Fr(1)
        rhs.append(e)
    for k in slopes:
        rows.append(_slope_row(k, deg))
        e = [Fr(0)] * NDATA
        e[5 + k + 2] = Fr(1)
        rhs.append(e)
    return _solve(rows, rhs)


def eval_functional(C, xi, nder=0):
    """Exact row r with (d^nder p / dxi^nder)(xi) = sum_d r[d] d[d]."""
    xi = Fr(xi)
    out = [Fr(0)] * NDATA
    for n, row in enumerate(C):
        if n < nder:
            continue
        f = Fr(1)
        for q in range(nder):
            f *= n - q
        w = f * xi ** (n - nder)
        for d in range(NDATA):
            out[d] += w * row[d]
    return out


def poly_tables():
    """All six stencils as float64 arrays of shape (9, 10) (zero-padded degree)."""
    out = {}
    for name in STENCILS:
        C = stencil_poly(name)
        T = np.zeros((9, NDATA))
        for n, row in enumerate(C):
            T[n] = [float(x) for x in row]
        out[name] = T
    return out


def gauss_legendre_unit(m):
    """Gauss-Legendre nodes on [-1/2, 1/2] and weights normalised to sum 1.

    Two, three and four points per face for orders 5, 7 and 9 (Sec. 3.3).
    """
    x, w = np.polynomial.legendre.leggauss(m)
    return 0.5 * x, 0.5 * w
