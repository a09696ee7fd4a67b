"""Pins of the oracle's wall boundaries (reflective slip wall, adiabatic no-slip
wall) and of the viscous collision time tau = mu / p (Sec. 4, Sec. 4.4, 4.9).

A reflective wall is the symmetry plane of a periodic problem twice as long
whose data are mirrored across it, so a wall run must equal the half of the
doubled periodic run (the periodic path does not use the ghost rule at all).
A closed box conserves mass and energy.  The viscous collision time must give
the Navier-Stokes shear viscosity: a small shear wave decays as
exp(-nu k^2 t), with or without no-slip walls.
"""
import numpy as np
import pytest

from oracle import (BC_NOSLIP, BC_PERIODIC, BC_REFLECTIVE, TAU_HGKS, TAU_NS, Oracle)
from paper_2508_13705_gb300 import inputs

def wall_impact_1d(n, gamma=1.4):
    """Gas at rho = p = 1 moving right at u = 1.5 + 0.2 sin(2 pi x) on [0,1]:
    a shock reflects off the right wall and a rarefaction leaves the left one
    from the first step.  Exact cell averages and slopes of the smooth data."""
    h = 1.0 / n
    xl = np.arange(n) * h
    xr = xl + h
    k = 2 * np.pi
    ubar = 1.5 + 0.2 * (np.cos(k * xl) - np.cos(k * xr)) / (k * h)
    ux = 0.2 * (np.sin(k * xr) - np.sin(k * xl)) / h
    # <u^2>: 2.25 + 0.6 <sin> + 0.04 <sin^2>
    s1 = (np.cos(k * xl) - np.cos(k * xr)) / (k * h)
    s2 = 0.5 - (np.sin(2 * k * xr) - np.sin(2 * k * xl)) / (4 * k * h)
    u2 = 2.25 + 0.6 * s1 + 0.04 * s2
    u2x = ((1.5 + 0.2 * np.sin(k * xr)) ** 2 - (1.5 + 0.2 * np.sin(k * xl)) ** 2) / h
    W = np.stack([np.ones(n), ubar, 1.0 / (gamma - 1) + 0.5 * u2])[:, None, :]
    Wx = np.stack([np.zeros(n), ux, 0.5 * u2x])[:, None, :]
    return W, Wx


def mirror_double(fields, axis, m, noslip=False):
    """Append the mirror image across the high end of ``axis`` (0: x, 1: y) to
    2-D SoA fields (W, Wx, Wy, Wx_line, Wy_line) or 1-D fields (W, Wx).
    Reflection maps q(x) to S q(-x): S reverses the normal momentum (every
    momentum for no-slip); a derivative along the normal takes one more sign;
    line data on lines across the mirror (Gauss nodes along the normal) are
    stored in reverse node order."""
    dim = 1 if len(fields) == 2 else 2
    nv = fields[0].shape[0] if dim == 1 else fields[0].shape[0]
    mom = [1 + axis] if not noslip else list(range(1, nv - 1))
    S = np.ones(nv)
    S[mom] = -1.0
    names = ("W", "Wx") if dim == 1 else ("W", "Wx", "Wy", "Wxl", "Wyl")
    out = []
    for name, f in zip(names, fields):
        dn = name in (("Wx", "Wxl") if axis == 0 else ("Wy", "Wyl"))
        sign = -S if dn else S
        line = name in ("Wxl", "Wyl")
        ax = f.ndim - 1 - axis  # x is the last axis, y the one before
        flip = np.flip(f, axis=ax)
        if line:
            if (axis == 0 and name == "Wyl") or (axis == 1 and name == "Wxl"):
                flip = np.flip(flip, axis=0)
            flip = flip * sign[None, :, None, None]
        else:
            flip = flip * sign.reshape((-1,) + (1,) * (f.ndim - 1))
        out.append(np.concatenate([f, flip], axis=ax))
    return out


@pytest.mark.parametrize("order", [5, 9])
def test_reflective_wall_1d_equals_mirrored_periodic(order):
    """Gas driven into one wall and away from the other, between two walls,
    vs the periodic problem on [0, 2] with the data mirrored about x = 1: the
    left halves agree to rounding over 40 steps, through the reflected shock
    and the HWENO-AO cells around it."""
    n = 100
    W, Wx = wall_impact_1d(n)
    kw = dict(tau_mode=TAU_HGKS)
    ow = Oracle(1, order, n, extent=(0, 1, 0, 1), bc=(BC_REFLECTIVE,) * 4, **kw)
    ow.set_state(W, Wx)
    Wp, Wxp = mirror_double([W, Wx], 0, 1)
    op = Oracle(1, order, 2 * n, extent=(0, 2, 0, 1), bc=(BC_PERIODIC,) * 4, **kw)
    op.set_state(Wp, Wxp)
    used_ao = False
    for _ in range(40):
        dt = op.compute_dt()
        ow.step(dt)
        op.step(dt)
        used_ao |= bool((ow.branch == 0).any())
    assert ow.flags == 0 and op.flags == 0 and used_ao
    for a, b in ((ow.W, op.W[..., :n]), (ow.Wx, op.Wx[..., :n]), (ow.sx, op.sx[..., :n + 1])):
        assert np.abs(a - b).max() <= 1e-11 * np.abs(b).max()


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("order", [5, 9])
def test_reflective_wall_2d_equals_mirrored_periodic(axis, order):
    """Seeded quadrant data with walls across ``axis`` (periodic along the
    other) vs the periodic problem doubled by mirroring across that axis
    (seed 3: a draw whose first steps stay physical under both wall pairs)."""
    nx, ny = 12, 10
    st = [a[..., :ny, :nx] for a in inputs.quadrants_2d(max(nx, ny), order, seed=3)]
    m = {5: 2, 7: 3, 9: 4}[order]
    rng = np.random.default_rng(5)
    # smooth random slopes so that every field and its mirror rule is exercised
    st = [st[0]] + [0.02 * rng.standard_normal(a.shape) for a in st[1:]]
    bc = [BC_PERIODIC] * 4
    bc[2 * axis] = bc[2 * axis + 1] = BC_REFLECTIVE
    kw = dict(tau_mode=TAU_HGKS)
    ow = Oracle(2, order, nx, ny, extent=(0, 1, 0, 1), bc=tuple(bc), **kw)
    ow.set_state(*st)
    dbl = mirror_double(st, axis, m)
    ext = (0, 2, 0, 1) if axis == 0 else (0, 1, 0, 2)
    op = Oracle(2, order, nx * (2 if axis == 0 else 1), ny * (2 if axis == 1 else 1), extent=ext, **kw)
    op.set_state(*dbl)
    for _ in range(3):
        dt = op.compute_dt()
        ow.step(dt)
        op.step(dt)
    assert ow.flags == 0 and op.flags == 0
    half = (Ellipsis, slice(0, nx)) if axis == 0 else (Ellipsis, slice(0, ny), slice(None))
    for a, b in ((ow.W, op.W), (ow.Wx, op.Wx), (ow.Wy, op.Wy), (ow.Wxl, op.Wxl), (ow.Wyl, op.Wyl)):
        bh = b[half]
        assert np.abs(a - bh).max() <= 1e-11 * max(1.0, np.abs(bh).max())


def test_closed_box_conserves_mass_and_energy():
    """Reflective walls on all four sides: no mass or energy crosses them."""
    n = 16
    st = inputs.quadrants_2d(n, 7, seed=0)
    o = Oracle(2, 7, n, n, extent=(0, 1, 0, 1), tau_mode=TAU_HGKS, bc=(BC_REFLECTIVE,) * 4)
    o.set_state(*st)
    m0 = o.W.sum(axis=(1, 2))
    for _ in range(15):
        o.step(o.compute_dt())
    assert o.flags == 0
    m1 = o.W.sum(axis=(1, 2))
    for v in (0, 3):
        assert abs(m1[v] - m0[v]) <= 1e-13 * abs(m0[v])


def shear_wave(nx, ny, order, A, walls):
    """v = A sin(k x) on a uniform gas at rest (rho = p = 1), k = 2 pi (periodic)
    or pi (walls at x = 0, 1), with exact cell averages and slopes."""
    m = {5: 2, 7: 3, 9: 4}[order]
    k = np.pi if walls else 2 * np.pi
    h = 1.0 / nx
    xl = np.arange(nx) * h
    xr = xl + h
    W = np.zeros((4, ny, nx))
    W[0] = 1.0
    W[2] = (A * (np.cos(k * xl) - np.cos(k * xr)) / (k * h))[None, :]
    s2 = A * A * (0.5 - (np.sin(2 * k * xr) - np.sin(2 * k * xl)) / (4 * k * h))
    W[3] = 1.0 / 0.4 + 0.5 * s2[None, :]
    Wx = np.zeros_like(W)
    Wx[2] = (A * (np.sin(k * xr) - np.sin(k * xl)) / h)[None, :]
    Wx[3] = (0.5 * A * A * (np.sin(k * xr) ** 2 - np.sin(k * xl) ** 2) / h)[None, :]
    return (W, Wx, np.zeros_like(W), np.repeat(Wx[None], m, axis=0), np.zeros((m, 4, ny, nx))), k, xl + 0.5 * h


@pytest.mark.parametrize("walls", [False, True])
def test_viscous_shear_wave_decays_at_nu_k2(walls):
    """tau = mu / p (Sec. 4) gives the shear viscosity mu: the amplitude of a
    small shear wave decays as exp(-nu k^2 t), nu = mu / rho, periodic or
    between no-slip walls; the error falls with the mesh."""
    mu, t_end = 0.01, 0.5
    errs = []
    for nx in (16, 32):
        st, k, xc = shear_wave(nx, 4, 5, 1e-3, walls)
        bc = (BC_NOSLIP, BC_NOSLIP, BC_PERIODIC, BC_PERIODIC) if walls else (BC_PERIODIC,) * 4
        o = Oracle(2, 5, nx, 4, extent=(0, 1, 0, 4.0 / nx), tau_mode=TAU_NS, bc=bc, mu=mu)
        o.set_state(*st)
        a0 = (st[0][2, 0] * np.sin(k * xc)).sum()
        o.run(t_end)
        assert o.flags == 0
        rate = -np.log((o.W[2, 0] * np.sin(k * xc)).sum() / a0) / t_end
        errs.append(abs(rate / (mu * k * k) - 1))
    assert errs[0] < 1e-2 and errs[1] < 0.6 * errs[0]


def test_viscous_time_step_limit():
    """dt = C min(h / (|U| + a), h^2 / (4 nu)): with a large viscosity the
    second bound decides."""
    n = 8
    st, _, _ = shear_wave(n, n, 5, 0.0, False)
    st = (st[0], st[1], st[2], st[3], st[4])
    mu = 0.5
    o = Oracle(2, 5, n, n, extent=(0, 1, 0, 1), tau_mode=TAU_NS, mu=mu, cfl=0.5)
    o.set_state(*st)
    h = 1.0 / n
    assert abs(o.compute_dt() - 0.5 * h * h / (4 * mu)) <= 1e-15


def test_initial_sigma_at_a_wall():
    """At t = 0 a wall face sees the adjacent cell and its mirror: Eq. 3.2 gives
    (2 Ma_n)^2 for the slip wall, plus (2 Ma_t)^2 for the no-slip wall."""
    n = 6
    u, v, p, rho, g = 0.3, -0.2, 1.0, 1.0, 1.4
    W = np.zeros((4, n, n))
    W[0], W[1], W[2] = rho, rho * u, rho * v
    W[3] = p / (g - 1) + 0.5 * rho * (u * u + v * v)
    z = np.zeros_like(W)
    zl = np.zeros((2, 4, n, n))
    a = np.sqrt(g * p / rho)
    for bc, want in ((BC_REFLECTIVE, (2 * u / a) ** 2), (BC_NOSLIP, (2 * u / a) ** 2 + (2 * v / a) ** 2)):
        o = Oracle(2, 5, n, n, extent=(0, 1, 0, 1), bc=(bc, bc, BC_PERIODIC, BC_PERIODIC))
        o.set_state(W, z, z, zl, zl)
        assert np.allclose(o.sx[:, 0], want, rtol=1e-14) and np.allclose(o.sx[:, n], want, rtol=1e-14)
        assert np.abs(o.sx[:, 1:n]).max() == 0.0
