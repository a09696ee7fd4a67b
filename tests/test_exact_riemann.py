"""Pins of the exact Riemann solver that the shock-tube and robustness tests
compare against: conservation of the exact solution, Riemann invariants
through the rarefaction fans, and the Rankine-Hugoniot jump conditions."""
import numpy as np
import pytest

import exact_riemann as er

DOUBLE_RAREFACTION = ((1.0, -2.0, 0.1), (1.0, 2.0, 0.1))  # Sec. 4.5: vacuum forms
SOD = ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
LAX = ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571))


def _cons(w, g):
    rho, u, p = w
    return np.array([rho, rho * u, p / (g - 1) + 0.5 * rho * u * u])


def _flux(w, g):
    rho, u, p = w
    E = p / (g - 1) + 0.5 * rho * u * u
    return np.array([rho * u, rho * u * u + p, u * (E + p)])


def _jumps(left, right, t, g, x0, x1, xs, n=4000):
    """Discontinuities of the sampled density (shock, contact), located by
    bisection between grid points where it changes by more than a smooth
    fan can over one spacing."""
    f = lambda x: er.sample(left, right, (np.atleast_1d(x) - xs) / t, g)[0]
    x = np.linspace(x0, x1, n + 1)
    r = f(x)
    out = []
    for k in np.nonzero(np.abs(np.diff(r)) > 50.0 * (x1 - x0) / n)[0]:
        a, b = x[k], x[k + 1]
        for _ in range(60):
            m = 0.5 * (a + b)
            if abs(f(m)[0] - r[k]) < abs(f(m)[0] - r[k + 1]):
                a = m
            else:
                b = m
        out.append(0.5 * (a + b))
    return out


def _integral(left, right, t, g, x0=0.0, x1=1.0, xs=0.5, cells=400, nq=8):
    """Composite Gauss quadrature of the conserved variables of the exact
    solution over [x0, x1] at time t, split at its discontinuities."""
    q, w = np.polynomial.legendre.leggauss(nq)
    edges = [x0] + _jumps(left, right, t, g, x0, x1, xs) + [x1]
    acc = np.zeros(3)
    for a, b in zip(edges[:-1], edges[1:]):
        h = (b - a) / cells
        xc = a + (np.arange(cells) + 0.5) * h
        for k in range(nq):
            x = xc + 0.5 * q[k] * h
            acc += 0.5 * w[k] * h * _cons(er.sample(left, right, (x - xs) / t, g), g).sum(axis=1)
    return acc


@pytest.mark.parametrize("left,right,t", [(*DOUBLE_RAREFACTION, 0.1), (*SOD, 0.2), (*LAX, 0.14)])
def test_exact_solution_conserves(left, right, t):
    """While no wave has reached the ends, d/dt of the integral of U equals
    the flux in at x0 minus the flux out at x1, both from the initial states."""
    g = 1.4
    U0 = 0.5 * _cons(left, g) + 0.5 * _cons(right, g)
    want = U0 + t * (_flux(left, g) - _flux(right, g))
    got = _integral(left, right, t, g)
    assert np.allclose(got, want, rtol=0, atol=2e-7), (got, want)


def test_double_rarefaction_generates_vacuum():
    assert er.generates_vacuum(*DOUBLE_RAREFACTION)
    assert not er.generates_vacuum(*SOD) and not er.generates_vacuum(*LAX)
    g, t = 1.4, 0.1
    a = np.sqrt(g * 0.1)
    tail = -2.0 + 2 * a / (g - 1)  # left fan tail speed
    x = 0.5 + np.array([0.5 * tail, 0.0, -0.5 * tail]) * t
    w = er.sample(*DOUBLE_RAREFACTION, (x - 0.5) / t, g)
    assert np.all(w[0] == 0.0) and np.all(w[2] == 0.0)


def test_riemann_invariant_through_left_fan():
    """u + 2a/(gamma-1) is constant through a left-facing rarefaction, and
    p / rho^gamma (isentropic)."""
    g = 1.4
    (rl, ul, pl), _ = DOUBLE_RAREFACTION
    al = np.sqrt(g * pl / rl)
    s = np.linspace(ul - al, ul + 2 * al / (g - 1), 50)[1:-1]
    rho, u, p = er.sample(*DOUBLE_RAREFACTION, s, g)
    a = np.sqrt(g * p / rho)
    assert np.allclose(u + 2 * a / (g - 1), ul + 2 * al / (g - 1), rtol=0, atol=1e-12)
    assert np.allclose(p / rho ** g, pl / rl ** g, rtol=1e-12)
    assert np.allclose(u - a, s, rtol=0, atol=1e-12)  # the fan is self-similar: u - a = x / t


def test_sod_shock_satisfies_rankine_hugoniot():
    g = 1.4
    ps, us = er.star_state(*SOD, g)
    rr, ur, pr = SOD[1]
    rs = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
    S = (rs * us - rr * ur) / (rs - rr)  # shock speed from the mass jump
    Wl, Wr = (rs, us, ps), (rr, ur, pr)
    jump_U = _cons(Wl, g) - _cons(Wr, g)
    jump_F = _flux(Wl, g) - _flux(Wr, g)
    assert np.allclose(jump_F, S * jump_U, rtol=1e-10, atol=1e-12)
