"""Pins of the oracle's kinetic part (Eq. 2.2-2.8, 2.11-2.12) against brute-force
quadrature of the Maxwellian and against the Euler equations."""
import itertools

import numpy as np
import pytest
from scipy import integrate

from oracle import Oracle, TAU_HGKS

G = 1.4


def cons1(r, u, p):
    return np.array([r, r * u, p / (G - 1) + 0.5 * r * u * u])


def cons2(r, u, v, p):
    return np.array([r, r * u, r * v, p / (G - 1) + 0.5 * r * (u * u + v * v)])


def euler_flux(W):
    if len(W) == 3:
        r, m, E = W
        u = m / r
        p = (G - 1) * (E - 0.5 * r * u * u)
        return np.array([m, m * u + p, u * (E + p)])
    r, mx, my, E = W
    u, v = mx / r, my / r
    p = (G - 1) * (E - 0.5 * r * (u * u + v * v))
    return np.array([mx, mx * u + p, mx * v, u * (E + p)])


def euler_flux_y(W):
    r, mx, my, E = W
    Wr = np.array([r, my, mx, E])
    F = euler_flux(Wr)
    return np.array([F[0], F[2], F[1], F[3]])


def jac(f, W, h=1e-6):
    J = np.zeros((len(W), len(W)))
    for k in range(len(W)):
        e = np.zeros(len(W))
        e[k] = h * max(1.0, abs(W[k]))
        J[:, k] = (f(W + e) - f(W - e)) / (2 * e[k])
    return J


# ------------------------------------------------------------------ moments

@pytest.mark.parametrize("dim", [1, 2])
def test_moments_against_quadrature(dim):
    o = Oracle(dim, 5, 4, 4)
    W = cons2(1.3, 0.4, -0.7, 0.8) if dim == 2 else cons1(1.3, 0.4, 0.8)
    mu, mv, mxi, fl = o.moments(W)
    assert fl == 0
    rho = W[0]
    U = W[1] / rho
    V = W[2] / rho if dim == 2 else 0.0
    p = 0.8
    lam = rho / (2 * p)
    s, w = np.polynomial.hermite.hermgauss(20)
    for n in range(10):
        full = (w * (U + s / np.sqrt(lam)) ** n).sum() / np.sqrt(np.pi)
        assert abs(mu[0, n] - full) <= 1e-12 * max(1, abs(full))
        g = lambda u: u ** n * np.sqrt(lam / np.pi) * np.exp(-lam * (u - U) ** 2)
        pos = integrate.quad(g, 0, np.inf, epsabs=1e-14, epsrel=1e-13)[0]
        neg = integrate.quad(g, -np.inf, 0, epsabs=1e-14, epsrel=1e-13)[0]
        assert abs(mu[1, n] - pos) <= 1e-10 * max(1, abs(pos))
        assert abs(mu[2, n] - neg) <= 1e-10 * max(1, abs(neg))
        assert abs(mu[1, n] + mu[2, n] - mu[0, n]) <= 1e-12 * max(1, abs(mu[0, n]))
        vv = (w * (V + s / np.sqrt(lam)) ** n).sum() / np.sqrt(np.pi)
        assert abs(mv[n] - vv) <= 1e-12 * max(1, abs(vv))
    # internal degrees of freedom: K = 3 (2-D) / 4 (1-D) for gamma = 1.4
    K = 3 if dim == 2 else 4
    nodes = [s / np.sqrt(lam)] * K
    ws = [w / np.sqrt(np.pi)] * K
    for c in range(3):
        acc = 0.0
        for idx in itertools.product(range(len(s)), repeat=K):
            xi2 = sum(nodes[k][i] ** 2 for k, i in enumerate(idx))
            acc += np.prod([ws[k][i] for k, i in enumerate(idx)]) * xi2 ** c
        assert abs(mxi[c] - acc) <= 1e-11 * max(1, acc)


@pytest.mark.parametrize("dim", [1, 2])
def test_micro_slope_solves_moment_system(dim):
    """<a> = b (Eq. 2.8): check the solution by an independent Gram matrix
    assembled from Gauss-Hermite quadrature of the Maxwellian."""
    o = Oracle(dim, 5, 4, 4)
    W = cons2(0.9, -0.3, 0.5, 1.7) if dim == 2 else cons1(0.9, -0.3, 1.7)
    rng = np.random.default_rng(3)
    b = rng.normal(size=len(W))
    a = o.micro_slope(W, b)
    rho, U = W[0], W[1] / W[0]
    V = W[2] / rho if dim == 2 else 0.0
    lam = rho / (2 * 1.7)
    K = 3 if dim == 2 else 4
    s, w = np.polynomial.hermite.hermgauss(8)
    x = s / np.sqrt(lam)
    wn = w / np.sqrt(np.pi)
    # xi^2 moments of the K internal components, and velocity nodes
    m_xi = [1.0, K / (2 * lam), K * (K + 2) / (4 * lam ** 2)]
    M = np.zeros((len(W), len(W)))
    us = U + x
    vs = V + x if dim == 2 else np.zeros(1)
    wv = wn if dim == 2 else np.ones(1)
    for iu, u in enumerate(us):
        for iv, v in enumerate(vs):
            # psi as polynomials in xi^2: value = c0 + c1 xi^2
            if dim == 2:
                psi = [(1, 0), (u, 0), (v, 0), (0.5 * (u * u + v * v), 0.5)]
            else:
                psi = [(1, 0), (u, 0), (0.5 * u * u, 0.5)]
            for i, (pi0, pi1) in enumerate(psi):
                for j, (pj0, pj1) in enumerate(psi):
                    e = pi0 * pj0 * m_xi[0] + (pi0 * pj1 + pi1 * pj0) * m_xi[1] + pi1 * pj1 * m_xi[2]
                    M[i, j] += wn[iu] * wv[iv] * rho * e
    assert np.allclose(M @ a, b, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------ fluxes

@pytest.mark.parametrize("tau_mode", [0, 1])
def test_uniform_state_gives_euler_flux_1d(tau_mode):
    o = Oracle(1, 5, 4, tau_mode=tau_mode)
    W = cons1(1.3, 0.7, 0.9)
    D = np.zeros((3, 3)); D[0] = W
    out, fl = o.point(D, D, 0.1)
    F = euler_flux(W)
    assert fl == 0
    assert np.allclose(out[0], 0.1 * F, rtol=1e-14, atol=1e-15)
    assert np.allclose(out[1], 0.05 * F, rtol=1e-14, atol=1e-15)
    for k in (2, 3, 4):
        assert np.allclose(out[k], W, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("tau_mode", [0, 1])
def test_uniform_state_gives_euler_flux_2d(tau_mode):
    o = Oracle(2, 5, 4, 4, tau_mode=tau_mode)
    W = cons2(0.8, -0.4, 1.1, 1.6)
    D = np.zeros((6, 4)); D[0] = W
    out, fl = o.point(D, D, 0.02)
    assert np.allclose(out[0], 0.02 * euler_flux(W), rtol=1e-14, atol=1e-16)
    assert np.allclose(out[2], W, rtol=1e-14)


def test_cauchy_kovalevskaya_1d():
    """tau = 0, equal smooth states: the fitted F_t (Eq. 2.20) and W_t (Eq. 2.29)
    equal the Euler time derivatives -A^2 W_x and -A W_x (A = dF/dW)."""
    o = Oracle(1, 5, 4)
    W = cons1(1.1, 0.35, 0.95)
    Wx = np.array([0.3, -0.2, 0.45])
    Wxx = np.array([-0.1, 0.05, 0.2])
    D = np.stack([W, Wx, Wxx])
    dt = 1e-2
    out, fl = o.point(D, D, dt)
    Fd, Fh, W0, Wh, Wd = out
    A = jac(euler_flux, W)
    F = (4 * Fh - Fd) / dt
    Ft = 4 * (Fd - 2 * Fh) / dt ** 2
    Wt = (4 * Wh - 3 * W0 - Wd) / dt
    assert np.allclose(W0, W, rtol=1e-14)
    assert np.allclose(F, euler_flux(W), rtol=1e-12)
    assert np.allclose(Ft, -A @ A @ Wx, rtol=1e-7, atol=1e-9)
    assert np.allclose(Wt, -A @ Wx, rtol=1e-7, atol=1e-9)


def test_cauchy_kovalevskaya_2d():
    o = Oracle(2, 7, 4, 4)
    W = cons2(1.1, 0.35, -0.6, 0.95)
    rng = np.random.default_rng(7)
    D = np.zeros((6, 4)); D[0] = W
    D[1:] = 0.3 * rng.normal(size=(5, 4))
    dt = 1e-2
    out, fl = o.point(D, D, dt)
    Fd, Fh, W0, Wh, Wd = out
    A = jac(euler_flux, W)
    B = jac(euler_flux_y, W)
    Wt_exact = -A @ D[1] - B @ D[3]
    Ft = 4 * (Fd - 2 * Fh) / dt ** 2
    Wt = (4 * Wh - 3 * W0 - Wd) / dt
    assert np.allclose(Wt, Wt_exact, rtol=1e-7, atol=1e-9)
    assert np.allclose(Ft, A @ Wt_exact, rtol=1e-7, atol=1e-9)


def test_kinetic_weighting_against_quadrature():
    """Different left/right states, no slopes, tau = 0: W(0) is the kinetic
    weighting Q0 = int_{u>0} psi g^l + int_{u<0} psi g^r (Eq. 2.7), and the
    flux is the Euler flux of Q0 (f = g0 when all slopes vanish)."""
    o = Oracle(1, 5, 4)
    Wl, Wr = cons1(1.0, 0.2, 1.0), cons1(0.4, -0.3, 0.5)
    Dl = np.zeros((3, 3)); Dl[0] = Wl
    Dr = np.zeros((3, 3)); Dr[0] = Wr
    out, _ = o.point(Dl, Dr, 0.01)
    K = 4

    def half(Wq, lo, hi):
        r, u0 = Wq[0], Wq[1] / Wq[0]
        p = (G - 1) * (Wq[2] - 0.5 * r * u0 * u0)
        lam = r / (2 * p)
        g = lambda u: r * np.sqrt(lam / np.pi) * np.exp(-lam * (u - u0) ** 2)
        q = lambda f: integrate.quad(lambda u: f(u) * g(u), lo, hi, epsabs=1e-14, epsrel=1e-13)[0]
        return np.array([q(lambda u: 1.0), q(lambda u: u),
                         q(lambda u: 0.5 * u * u) + 0.5 * K / (2 * lam) * q(lambda u: 1.0)])

    Q0 = half(Wl, 0, np.inf) + half(Wr, -np.inf, 0)
    assert np.allclose(out[2], Q0, rtol=1e-10)
    assert np.allclose(out[0] / 0.01, euler_flux(Q0), rtol=1e-10)


def test_collision_terms_cancel_for_equal_states():
    """tau > 0 (HGKS rule) with equal states and no slopes: every non-equilibrium
    term of Eq. 2.6 cancels and the flux stays the Euler flux."""
    o = Oracle(1, 9, 4, tau_mode=TAU_HGKS)
    W = cons1(2.0, -0.5, 3.0)
    D = np.zeros((3, 3)); D[0] = W
    out, _ = o.point(D, D, 0.3)
    assert np.allclose(out[0], 0.3 * euler_flux(W), rtol=1e-13)
