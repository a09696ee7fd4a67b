"""Pins of the oracle's HWENO-AO branch (Eq. 3.11-3.17, 3.19), of the
e^{-t/tau} terms of the third-order distribution (Eq. 2.6) with their time
integrals (Eq. 2.15), and of the temporal order of the two-stage S2O4 update
(Eq. 2.13-2.14).  Every expected value comes from an independent route:
adaptive quadrature, a closed form the definitions force, or a limit."""
import numpy as np
import pytest
from scipy import integrate

from oracle import TAU_HGKS, Oracle, coeffs
from paper_2508_13705_gb300 import inputs

G = 1.4


def _poly_val(p, x, nd=0):
    """d^nd/dxi^nd of sum_n p[n] xi^n at x."""
    return np.polynomial.polynomial.polyval(x, np.polynomial.polynomial.polyder(p, nd) if nd else p)


# ------------------------------------------------------------------ Eq. 3.13

@pytest.mark.parametrize("deg", [2, 4])
def test_smoothness_indicator_against_quadrature(deg):
    """beta = sum_{q=1}^{deg} dx^{2q-1} int_{cell} (d^q p / dx^q)^2 dx, taken by
    adaptive quadrature in physical coordinates on a cell of width dx = 0.37
    around x_i = 1.3, equals the oracle's value for the same polynomial in the
    unit coordinate xi = (x - x_i) / dx."""
    rng = np.random.default_rng(deg)
    o = Oracle(1, 5, 4)
    dx, xi0 = 0.37, 1.3
    for _ in range(5):
        c = rng.normal(size=deg + 1)  # coefficients in xi
        # the same polynomial in x: p(x) = sum_n c_n ((x - xi0) / dx)^n
        px = np.polynomial.Polynomial(c)(np.polynomial.Polynomial([-xi0 / dx, 1.0 / dx]))
        beta = 0.0
        for q in range(1, deg + 1):
            dq = px.deriv(q)
            val = integrate.quad(lambda x: dq(x) ** 2, xi0 - dx / 2, xi0 + dx / 2, epsabs=0, epsrel=1e-13)[0]
            beta += dx ** (2 * q - 1) * val
        assert abs(o.smoothness(c, deg) - beta) <= 1e-11 * max(1.0, beta)


# ------------------------------------------------------------------ Eq. 3.11-3.17, 3.19

TABS = coeffs.poly_tables()


def _data_of_poly(c):
    """d = [Qbar_{i-2..i+2}, dx Qx_{i-2..i+2}] of the polynomial sum c_n xi^n
    (exact cell averages and averaged slopes on the unit cells)."""
    P = np.polynomial.Polynomial(c)
    I = P.integ()
    avg = [I(k + 0.5) - I(k - 0.5) for k in range(-2, 3)]
    slo = [P(k + 0.5) - P(k - 0.5) for k in range(-2, 3)]
    return np.array(avg + slo)


def _scaled(st, d, alpha):
    p = TABS[st] @ d
    p[1:] *= alpha
    p[0] = d[2] + alpha * (p[0] - d[2])
    return p


def test_ao_equal_dffs_reproduce_scaled_quadratic():
    """Quadratic data with sigma only on the two faces of cell i: the sums of
    Eq. 3.3 are equal for S0, S1, S2 and r5, so every DFF is thr / A.  All four
    stencil polynomials reproduce the quadratic, their DFF-scaled forms are
    equal, and Eq. 3.17 must return that common polynomial whatever the
    nonlinear weights are."""
    o = Oracle(1, 9, 8)
    c = np.array([0.7, -0.4, 0.9])
    d = _data_of_poly(c)
    sig = np.array([0.0, 0.0, 0.7, 0.8, 0.0, 0.0])
    poly, br = o.recon(d, sig)
    assert br == 0  # HWENO-AO branch
    alpha = 1.0 / 1.5
    want = np.zeros(9)
    want[:3] = c * alpha
    want[0] = d[2] + alpha * (c[0] - d[2])
    assert np.allclose(poly, want, rtol=0, atol=1e-14)


def test_ao_weights_sum_to_one_preserve_cell_average():
    """Every stencil keeps the own cell average, so Eq. 3.17 keeps it exactly
    when the normalised weights of Eq. 3.16 sum to one: the AO polynomial's
    mean over the cell equals Qbar_i for arbitrary data and unequal DFFs."""
    rng = np.random.default_rng(11)
    o = Oracle(1, 9, 8)
    for _ in range(20):
        d = rng.normal(size=10)
        sig = rng.uniform(0.0, 0.9, size=6)
        sig[2] += 0.6
        poly, br = o.recon(d, sig)
        assert br == 0
        mean = sum(poly[n] * 2 * 0.5 ** (n + 1) / (n + 1) for n in range(0, 9, 2))
        assert abs(mean - d[2]) <= 1e-13 * max(1.0, np.abs(d).max())


def test_ao_large_epsilon_gives_scaled_r5():
    """With epsilon far above every smoothness indicator the WENO-Z weights of
    Eq. 3.14 equal the linear weights, and Eq. 3.17 collapses to the big
    stencil's polynomial (Eq. 3.11), here its DFF-scaled form (Eq. 3.19)."""
    rng = np.random.default_rng(5)
    o = Oracle(1, 9, 8, weno_eps=1e30)
    for _ in range(10):
        d = rng.normal(size=10)
        sig = rng.uniform(0.0, 0.5, size=6)
        sig[3] += 0.8
        poly, br = o.recon(d, sig)
        assert br == 0
        A_r5 = sig[1] + sig[2] + sig[3] + sig[4]
        want = _scaled("r5", d, min(1.0, 1.0 / A_r5))
        assert np.allclose(poly, want, rtol=0, atol=1e-13 * max(1.0, np.abs(d).max()))


def test_ao_eno_limit_picks_the_smooth_substencil():
    """A step between cells i and i+1 with cells i-1 and i flat: the DFF-scaled
    S0 polynomial is the constant Qbar_i, so beta_0 = 0 while the other
    indicators are O(1); the WENO-Z weight of S0 then exceeds the others by
    (tau_Z / eps)^2 and Eq. 3.17 returns the constant to rounding."""
    o = Oracle(1, 9, 8)
    d = np.array([0.3, 1.0, 1.0, 2.0, 2.1, 0.4, 0.0, -0.2, 0.0, 0.5])
    for sig in ([0.0, 0.1, 0.2, 1.5, 0.1, 0.0], [0.3, 0.6, 0.9, 2.5, 0.4, 0.2]):
        poly, br = o.recon(d, np.array(sig))
        assert br == 0
        want = np.zeros(9)
        want[0] = 1.0
        assert np.allclose(poly, want, rtol=0, atol=1e-12)


# ------------------------------------------------------------------ Eq. 2.6, 2.15

K1 = (3.0 - G) / (G - 1.0)  # internal degrees of freedom of the 1-D model


def _cons(r, u, p):
    return np.array([r, r * u, p / (G - 1) + 0.5 * r * u * u])


def _prim(W):
    r, u = W[0], W[1] / W[0]
    p = (G - 1) * (W[2] - 0.5 * r * u * u)
    return r, u, p


def _vint(W, lo, hi, pw, a=None):
    """int_{lo<u<hi} u^pw psi_i (a . (1, u, (u^2+xi^2)/2)) g dXi for the 1-D
    Maxwellian of W, i = 0..2, with psi = (1, u, (u^2 + xi^2)/2).  The K internal
    components are integrated in closed form (Gaussian moments of xi^2), the
    velocity u by adaptive quadrature."""
    r, U, p = _prim(W)
    lam = r / (2 * p)
    mxi = [1.0, K1 / (2 * lam), K1 * (K1 + 2) / (4 * lam ** 2)]
    a = np.array([1.0, 0.0, 0.0]) if a is None else a

    def psi(i, u):  # coefficients of (xi^2)^0, (xi^2)^1
        return [(1.0, 0.0), (u, 0.0), (0.5 * u * u, 0.5)][i]

    def integrand(u, i):
        s0, s1 = psi(i, u)
        b0, b1 = a[0] + a[1] * u + 0.5 * a[2] * u * u, 0.5 * a[2]
        poly = s0 * b0 * mxi[0] + (s0 * b1 + s1 * b0) * mxi[1] + s1 * b1 * mxi[2]
        return u ** pw * poly * r * np.sqrt(lam / np.pi) * np.exp(-lam * (u - U) ** 2)

    return np.array([integrate.quad(integrand, lo, hi, args=(i,), epsabs=1e-15, epsrel=1e-13, limit=200)[0]
                     for i in range(3)])


def _slope(W, b):
    """Micro-slope a with <a> = b (Eq. 2.8), from a quadrature Gram matrix."""
    G_ = np.stack([_vint(W, -np.inf, np.inf, 0, e) for e in np.eye(3)], axis=1)
    return np.linalg.solve(G_, b)


def test_time_integrals_against_velocity_quadrature():
    """Unequal left and right states with first and second slopes, HGKS
    collision time tau > 0.  The distribution of Eq. 2.6 (g^l with u > 0 and
    a^l, g^r with u < 0 and a^r) is built in velocity space: micro-slopes from
    quadrature Gram matrices, Q0 and its derivatives by half-range quadrature
    (Eq. 2.7), the compatibility conditions of Eq. 2.8.  Its moments at
    t = 0, dt/2, dt and its flux integrated over [0, delta] by adaptive
    quadrature in t (the t^2 a_tt term kept in the state, left out of the
    flux integral) must equal the oracle's closed-form time coefficients."""
    Wl, Wr = _cons(1.0, 0.2, 1.0), _cons(0.55, -0.15, 0.6)
    Dl = np.stack([Wl, [0.3, -0.2, 0.5], [-0.4, 0.3, 0.2]])
    Dr = np.stack([Wr, [-0.1, 0.25, -0.3], [0.2, -0.1, 0.6]])
    dt = 0.05
    o = Oracle(1, 5, 4, tau_mode=TAU_HGKS)
    out, fl = o.point(Dl, Dr, dt)
    assert fl == 0
    pl, pr = _prim(Wl)[2], _prim(Wr)[2]
    tau = 0.05 * dt + abs(pl - pr) / (pl + pr) * dt
    inf = np.inf
    a1l, a11l = _slope(Wl, Dl[1]), _slope(Wl, Dl[2])
    a1r, a11r = _slope(Wr, Dr[1]), _slope(Wr, Dr[2])
    Q0 = _vint(Wl, 0, inf, 0) + _vint(Wr, -inf, 0, 0)
    dQ = _vint(Wl, 0, inf, 0, a1l) + _vint(Wr, -inf, 0, 0, a1r)
    ddQ = _vint(Wl, 0, inf, 0, a11l) + _vint(Wr, -inf, 0, 0, a11r)
    a1 = _slope(Q0, dQ)
    a11 = _slope(Q0, ddQ)
    A = _slope(Q0, -_vint(Q0, -inf, inf, 1, a1))
    a1t = _slope(Q0, -_vint(Q0, -inf, inf, 1, a11))
    att = _slope(Q0, -_vint(Q0, -inf, inf, 1, a1t))

    def terms(pw):
        return dict(g0=_vint(Q0, -inf, inf, pw), A=_vint(Q0, -inf, inf, pw, A),
                    att=_vint(Q0, -inf, inf, pw, att), a1u=_vint(Q0, -inf, inf, pw + 1, a1),
                    a1tu=_vint(Q0, -inf, inf, pw + 1, a1t),
                    gl=_vint(Wl, 0, inf, pw), glu=_vint(Wl, 0, inf, pw + 1, a1l),
                    gr=_vint(Wr, -inf, 0, pw), gru=_vint(Wr, -inf, 0, pw + 1, a1r))

    def moments(T, t, with_tt):
        e = np.exp(-t / tau)
        return (T["g0"] + t * T["A"] + (0.5 * t * t * T["att"] if with_tt else 0.0)
                - tau * (T["a1u"] + T["A"]) - tau * t * (T["a1tu"] + T["att"])
                - e * T["g0"] + e * t * T["a1u"]
                + e * T["gl"] - e * t * T["glu"] + e * T["gr"] - e * t * T["gru"])

    S = terms(0)
    for k, t in enumerate((0.0, 0.5 * dt, dt)):
        assert np.allclose(out[2 + k], moments(S, t, True), rtol=1e-10, atol=1e-12)
    Fl = terms(1)
    for k, delta in enumerate((dt, 0.5 * dt)):
        F = integrate.quad_vec(lambda t: moments(Fl, t, False), 0.0, delta, epsabs=1e-16, epsrel=1e-12)[0]
        assert np.allclose(out[k], F, rtol=1e-9, atol=1e-14), (k, out[k], F)


# ------------------------------------------------------------------ Eq. 2.13-2.14

def _temporal_orders(order, flux_tt=0, N=80, t_end=0.4):
    sols = []
    for dt in (0.01, 0.005, 0.0025, 0.00125):
        o = Oracle(1, order, N, extent=(0, 2, 0, 1))
        o.P.flux_tt = flux_tt
        o.set_state(*inputs.density_wave_1d(N))
        o.run(t_end, dt_fn=lambda s, dt=dt: dt)
        assert o.flags == 0 and abs(o.t - t_end) < 1e-12
        sols.append(o.W.ravel().copy())
    e = np.array([np.abs(sols[k] - sols[k + 1]).mean() for k in range(3)])
    return e, np.log2(e[:-1] / e[1:])


@pytest.mark.parametrize("order", [7, 9])
def test_s2o4_is_fourth_order_in_time(order):
    """Fixed mesh (N = 80 on [0, 2], tau = 0, the density wave of Sec. 4.1),
    dt halved three times from 0.01 (CFL 0.87 to 0.11): successive differences
    of the solutions at t = 0.4 isolate the temporal error, whose observed
    order must be 4 (Eq. 2.13-2.14).  (At order 5 a mixed space-time term,
    linear in dt and of size dt h^4.6, shows below about 1e-11 at this mesh;
    it is invisible at orders 7 and 9.)"""
    e, orders = _temporal_orders(order)
    assert np.all(np.abs(orders - 4.0) < 0.2), (e, orders)


def test_literal_quadratic_flux_term_is_second_order_in_time():
    """The same sequence with the t^2/2 a_tt g0 term kept in the flux
    integral: the linear fit of Eq. 2.19-2.20 then leaves an O(dt^3) local
    error and the observed temporal order drops to 2, which singles out the
    reading of the flux integral used everywhere else."""
    e, orders = _temporal_orders(7, flux_tt=1)
    assert abs(orders[-1] - 2.0) < 0.2, (e, orders)
