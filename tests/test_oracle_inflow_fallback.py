"""Pins of the inflow boundary sides (the supersonic inflow and the exact
shock motion of Sec. 4.8) and of the flagged first-order fallback at face
points, on the oracle: inflow of the boundary's own state against the
transmissive rule, the split wall's limit against the slip wall, the Mach 10
shock translating at its exact speed between moving inflow splits (with a
wrong speed as the control that the pin sees the split), the fallback's face
flux against the Euler flux in closed form, and the first steps of the double
Mach reflection."""
import numpy as np
import pytest

from oracle import BC_INFLOW, BC_INFLOW_REFLECTIVE, BC_REFLECTIVE, BC_TRANSMISSIVE, TAU_HGKS, Oracle
from paper_2508_13705_gb300 import inputs

G = 1.4


def _pressure(W):
    return (G - 1) * (W[3] - 0.5 * (W[1] ** 2 + W[2] ** 2) / W[0])


def _free_stream_with_bump(n, order, seed=0):
    """rho = 1, u = 0.3, v = -0.7, p = 1 with random density and pressure
    changes in the central 8 x 8 cells (zero slopes); returns the state and
    the conservative free stream."""
    rng = np.random.default_rng(seed)
    rho = np.ones((n, n))
    p = np.ones((n, n))
    c = slice(n // 2 - 4, n // 2 + 4)
    rho[c, c] += 0.3 * rng.random((8, 8))
    p[c, c] += 0.3 * rng.random((8, 8))
    W = np.stack([rho, 0.3 * rho, -0.7 * rho, p / (G - 1) + 0.5 * rho * (0.09 + 0.49)])
    m = {5: 2, 7: 3, 9: 4}[order]
    z = np.zeros_like(W)
    free = np.array([1.0, 0.3, -0.7, 1.0 / (G - 1) + 0.5 * 0.58])
    return (W, z, z.copy(), np.zeros((m, 4, n, n)), np.zeros((m, 4, n, n))), free


@pytest.mark.parametrize("order", [5, 9])
def test_inflow_of_the_boundary_state_equals_transmissive(order):
    """While the flow next to every side is the undisturbed free stream (zero
    slopes), the transmissive ghost cell and an inflow ghost cell holding that
    free stream are the same cell, with the same ghost sigma: one step agrees
    bitwise.  A ghost state in the wrong variable order, on the wrong side or
    with non-zero slopes would not."""
    n = 40
    st, free = _free_stream_with_bump(n, order)
    res = []
    for bc in ((BC_TRANSMISSIVE,) * 4, (BC_INFLOW,) * 4):
        o = Oracle(2, order, n, n, tau_mode=TAU_HGKS, bc=bc, bc_state=np.broadcast_to(free, (4, 2, 4)))
        o.set_state(*st)
        o.step(o.compute_dt())
        assert o.flags == 0
        res.append(o.get_state())
    for f in ("W", "Wx", "Wy", "Wx_line", "Wy_line", "sigma_x", "sigma_y"):
        assert np.array_equal(res[0][f], res[1][f]), f
    assert not np.array_equal(res[0]["W"], st[0])  # the step moved the bump


def test_split_wall_beyond_minus_infinity_is_the_slip_wall():
    """CGKS_BC_INFLOW_REFLECTIVE with its split point at -infinity is a slip
    wall along the whole side (ghost cells and ghost sigma): three steps of
    quadrant data between two such sides agree bitwise with the wall run."""
    nx, ny, order = 12, 10, 9
    st = [a[..., :ny, :nx] for a in inputs.quadrants_2d(12, order, seed=3)]
    rng = np.random.default_rng(5)
    st = [st[0]] + [0.02 * rng.standard_normal(a.shape) for a in st[1:]]
    split = np.zeros((4, 2))
    split[2:, 0] = -1e30
    res = []
    for bc in ((0, 0, BC_REFLECTIVE, BC_REFLECTIVE), (0, 0, BC_INFLOW_REFLECTIVE, BC_INFLOW_REFLECTIVE)):
        o = Oracle(2, order, nx, ny, tau_mode=TAU_HGKS, bc=bc, bc_split=split)
        o.set_state(*st)
        for _ in range(3):
            o.step(0.002)
        assert o.flags == 0
        res.append(o.get_state())
    for f in ("W", "Wx", "Wy", "Wx_line", "Wy_line", "sigma_x", "sigma_y"):
        assert np.array_equal(res[0][f], res[1][f]), f


def _exact_mass(t, xa, H, n=200000):
    """Mass of the translated Mach 10 shock in [0,1] x [0,H]: post-shock
    density 8 left of x = xa + (y + 20 t) / sqrt 3, 1.4 right of it."""
    y = (np.arange(n) + 0.5) * H / n
    L = np.clip(xa + (y + 20.0 * t) / np.sqrt(3.0), 0.0, 1.0)
    return (8.0 * L + 1.4 * (1.0 - L)).mean() * H


def _shock_rows(rho, nx):
    """x where each row's density first falls through 4.7 (linear between centres)."""
    xs = []
    for r in rho:
        k = int(np.nonzero(r < 4.7)[0][0])
        xs.append((k - 0.5 + (r[k - 1] - 4.7) / (r[k - 1] - r[k])) / nx)
    return np.array(xs)


def test_oblique_shock_translates_at_its_exact_speed():
    """The Mach 10 shock of Sec. 4.8 between inflow sides whose splits follow
    its exact position: after 16 steps the mass gained (the flux through the
    sides) is the exact one within 1.5 %, and the front sits within 1.5 cells
    of the exact line in every row.  Holding the splits still (speed 0), the
    mass is 5 % off and the front bends by 5 cells at the sides."""
    nx, ny, xa, H, t_end = 48, 24, 0.3, 0.5, 0.012
    dm_exact = _exact_mass(t_end, xa, H) - _exact_mass(0.0, xa, H)
    yc = (np.arange(ny) + 0.5) * H / ny
    x_exact = xa + (yc + 20.0 * t_end) / np.sqrt(3.0)
    out = {}
    for speed in (inputs.SHOCK_SPEED_X, 0.0):
        st, kw = inputs.oblique_shock(nx, ny, 5, xa=xa, height=H, speed=speed)
        o = Oracle(2, 5, nx, ny, tau_mode=TAU_HGKS, cfl=0.5, pt_fallback=1, **kw)
        o.set_state(*st)
        m0 = o.W[0].sum() * o.dx * o.dy
        o.run(t_end, max_steps=200)
        assert o.flags == 0 and o.W[0].min() > 0 and _pressure(o.W).min() > 0
        dm = o.W[0].sum() * o.dx * o.dy - m0
        out[speed] = (abs(dm / dm_exact - 1.0), np.abs(_shock_rows(o.W[0], nx) - x_exact).max() * nx)
    good, still = out[inputs.SHOCK_SPEED_X], out[0.0]
    assert good[0] < 0.015 and good[1] < 1.5, good
    assert still[0] > 0.05 and still[1] > 4.0, still


def test_fallback_is_off_by_default_and_idle_on_smooth_data():
    """With nothing non-physical the fallback changes no bit, and counts 0."""
    n, order = 16, 7
    st = inputs.density_wave_2d(n, order)
    res = []
    for pf in (0, 1):
        o = Oracle(2, order, n, n, extent=(0, 2, 0, 2), tau_mode=TAU_HGKS, pt_fallback=pf)
        o.set_state(*st)
        for _ in range(2):
            o.step(0.01)
        assert o.flags == 0 and o.fallbacks == 0
        res.append(o.get_state())
    for f in res[0]:
        assert np.array_equal(res[0][f], res[1][f]), f


def test_fallback_face_flux_is_the_euler_flux_of_the_cell_average():
    """1-D gas at rest (rho 1, p 1e-3) with energy slopes -10, -10, 10, 10 in
    cells 6..9: the order-5 reconstruction drives both sides of face 8 to a
    negative pressure (the kinetic evaluation fails without the fallback).
    With it, both sides take their cells' common average and zero
    derivatives, so the face sees one equilibrium state: F(dt) and F(dt/2)
    are dt and dt/2 times its Euler flux (0, p, 0), and W(0), W(dt/2), W(dt)
    the state itself."""
    N, f, dt, p = 16, 8, 1e-3, 1e-3
    W = np.zeros((3, 1, N))
    W[0] = 1.0
    W[2] = p / (G - 1)
    Wx = np.zeros((3, 1, N))
    Wx[2, 0, f - 2:f + 2] = (-10.0, -10.0, 10.0, 10.0)
    flags = []
    for pf in (0, 1):
        o = Oracle(1, 5, N, extent=(0, 1, 0, 1), tau_mode=TAU_HGKS, bc=(1, 1, 1, 1), pt_fallback=pf)
        o.set_state(W, Wx)
        out, _ = o.faces(dt)
        flags.append(o.flags)
    assert flags[0] != 0 and flags[1] == 0
    assert o.fallbacks >= 2
    face = out[:, :, 0, f]
    assert np.array_equal(face[0], np.array([0.0, p * dt, 0.0]))
    assert np.array_equal(face[1], np.array([0.0, p * dt / 2, 0.0]))
    for k in (2, 3, 4):
        assert np.array_equal(face[k], W[:, 0, f])


def test_double_mach_reflection_first_steps():
    """Sec. 4.8 at 48 x 12: without the fallback the staircase front of the
    Mach 10 shock drives stage-2 face states ahead of it to negative pressure
    in step 1 (the scheme's own reconstruction, whatever the boundaries: the
    transmissive run fails alike); with it, the first 5 steps stay positive."""
    nx, ny, order = 48, 12, 5
    st, kw = inputs.double_mach(nx, ny, order)
    for bc in (kw["bc"], (BC_TRANSMISSIVE,) * 4):
        o = Oracle(2, order, nx, ny, tau_mode=TAU_HGKS, cfl=0.5, **dict(kw, bc=bc))
        o.set_state(*st)
        o.step(o.compute_dt())
        assert o.flags != 0
    o = Oracle(2, order, nx, ny, tau_mode=TAU_HGKS, cfl=0.5, pt_fallback=1, **kw)
    o.set_state(*st)
    for _ in range(5):
        o.step(o.compute_dt())
        assert o.flags == 0 and o.W[0].min() > 0 and _pressure(o.W).min() > 0
    assert o.fallbacks > 0
