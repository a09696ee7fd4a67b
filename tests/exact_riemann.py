"""Exact solution of the 1-D Euler Riemann problem (ideal gas), used as a pin.

Textbook construction: the star-region pressure p* solves
f_L(p*) + f_R(p*) + (u_R - u_L) = 0, where f_K is the shock (Rankine-Hugoniot)
branch for p* > p_K and the rarefaction (isentropic) branch otherwise; it is
found by Newton iteration.  The self-similar solution is then sampled at x/t.
When 2 (a_L + a_R) / (gamma - 1) <= u_R - u_L no p* > 0 exists: the two
rarefactions separate and leave a vacuum between their tails.
"""
import numpy as np


def _f(p, rho, pk, gamma):
    a = np.sqrt(gamma * pk / rho)
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        s = np.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    r = (p / pk) ** ((gamma - 1.0) / (2.0 * gamma))
    return 2.0 * a / (gamma - 1.0) * (r - 1.0), (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma)) / (rho * a)


def star_state(left, right, gamma=1.4):
    rl, ul, pl = left
    rr, ur, pr = right
    p = max(1e-8, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dl = _f(p, rl, pl, gamma)
        fr, dr = _f(p, rr, pr, gamma)
        g = fl + fr + ur - ul
        pn = max(1e-12, p - g / (dl + dr))
        if abs(pn - p) < 1e-14 * (p + pn):
            p = pn
            break
        p = pn
    fl, _ = _f(p, rl, pl, gamma)
    fr, _ = _f(p, rr, pr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def _fan_left(left, s, g):
    rl, ul, pl = left
    al = np.sqrt(g * pl / rl)
    c = 2 / (g + 1) + (g - 1) / ((g + 1) * al) * (ul - s)
    return (rl * c ** (2 / (g - 1)), 2 / (g + 1) * (al + (g - 1) / 2 * ul + s), pl * c ** (2 * g / (g - 1)))


def _fan_right(right, s, g):
    rr, ur, pr = right
    ar = np.sqrt(g * pr / rr)
    c = 2 / (g + 1) - (g - 1) / ((g + 1) * ar) * (ur - s)
    return (rr * c ** (2 / (g - 1)), 2 / (g + 1) * (-ar + (g - 1) / 2 * ur + s), pr * c ** (2 * g / (g - 1)))


def generates_vacuum(left, right, gamma=1.4):
    """Pressure-positivity condition fails: the two rarefactions separate."""
    al, ar = np.sqrt(gamma * left[2] / left[0]), np.sqrt(gamma * right[2] / right[0])
    return 2 * (al + ar) / (gamma - 1) <= right[1] - left[1]


def _sample_vacuum(left, right, xi, g):
    """Two rarefactions whose tails, u_L + 2a_L/(g-1) and u_R - 2a_R/(g-1),
    bound a vacuum (rho = p = 0)."""
    rl, ul, pl = left
    rr, ur, pr = right
    al, ar = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    sl, sr = ul + 2 * al / (g - 1), ur - 2 * ar / (g - 1)
    out = np.zeros((3, len(xi)))
    for n, s in enumerate(xi):
        if s <= ul - al:
            out[:, n] = left
        elif s < sl:
            out[:, n] = _fan_left(left, s, g)
        elif s <= sr:
            out[:, n] = (0.0, s, 0.0)
        elif s < ur + ar:
            out[:, n] = _fan_right(right, s, g)
        else:
            out[:, n] = right
    return out


def sample(left, right, xi, gamma=1.4):
    """(rho, u, p) at similarity coordinates xi = (x - x0) / t (array)."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    xi = np.atleast_1d(np.asarray(xi, dtype=float))
    if generates_vacuum(left, right, g):
        return _sample_vacuum(left, right, xi, g)
    ps, us = star_state(left, right, gamma)
    al, ar = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    out = np.zeros((3, len(xi)))
    for n, s in enumerate(xi):
        if s <= us:  # left of contact
            if ps > pl:  # left shock
                sl = ul - al * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s <= sl:
                    out[:, n] = (rl, ul, pl)
                else:
                    r = rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1))
                    out[:, n] = (r, us, ps)
            else:  # left rarefaction
                ast = al * (ps / pl) ** ((g - 1) / (2 * g))
                if s <= ul - al:
                    out[:, n] = (rl, ul, pl)
                elif s >= us - ast:
                    out[:, n] = (rl * (ps / pl) ** (1 / g), us, ps)
                else:
                    out[:, n] = _fan_left(left, s, g)
        else:  # right of contact
            if ps > pr:
                sr = ur + ar * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s >= sr:
                    out[:, n] = (rr, ur, pr)
                else:
                    r = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
                    out[:, n] = (r, us, ps)
            else:
                ast = ar * (ps / pr) ** ((g - 1) / (2 * g))
                if s >= ur + ar:
                    out[:, n] = (rr, ur, pr)
                elif s <= us + ast:
                    out[:, n] = (rr * (ps / pr) ** (1 / g), us, ps)
                else:
                    out[:, n] = _fan_right(right, s, g)
    return out


def cell_average_rho(left, right, nx, t, x0=0.0, x1=1.0, xs=0.5, gamma=1.4, nq=16):
    """Cell averages of the exact density (Gauss quadrature in each cell)."""
    dx = (x1 - x0) / nx
    q, w = np.polynomial.legendre.leggauss(nq)
    xc = x0 + (np.arange(nx) + 0.5) * dx
    acc = np.zeros(nx)
    for k in range(nq):
        x = xc + 0.5 * q[k] * dx
        acc += 0.5 * w[k] * sample(left, right, (x - xs) / t, gamma)[0]
    return acc
