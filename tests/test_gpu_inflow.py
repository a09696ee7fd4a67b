"""Inflow boundary sides and the first-order point fallback on the GPU
(Sec. 4.8): per-step parity with the FP64 oracle on the double Mach
reflection and on the translating Mach 10 shock (the stage times of the
moving splits and the fallback decisions included: the counts match
exactly), then the double Mach reflection on the paper's 960 x 240 mesh to
t = 0.2."""
import numpy as np
import pytest

import oracle
from paper_2508_13705_gb300 import cgks, inputs
from test_gpu_parity import FIELDS_2D, compare

pytestmark = pytest.mark.gpu
G = 1.4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2508_13705_gb300 import build
    build.build()
    oracle.build()


def _pressure(W):
    return (G - 1) * (W[3] - 0.5 * (W[1] ** 2 + W[2] ** 2) / W[0])


def per_step_timed(order, nx, ny, st, kw, steps, what, precision=cgks.FP64):
    """Both sides start every step from the oracle's state and time; the GPU's
    fallback count (reset by set_state) equals the oracle's for that step."""
    common = dict(tau_mode=cgks.TAU_HGKS, cfl=0.5, pt_fallback=1, **kw)
    o = oracle.Oracle(2, order, nx, ny, **common)
    o.set_state(*st)
    s = cgks.Solver(2, order, nx, ny, precision=precision, **common)
    total = 0
    for k in range(steps):
        g0 = o.get_state()
        s.set_state(g0["W"], g0["Wx"], g0["Wy"], g0["Wx_line"], g0["Wy_line"], g0["sigma_x"], g0["sigma_y"])
        s.set_time(o.t)
        dt = o.compute_dt()
        before = o.fallbacks
        s.step(dt)
        s.sync()
        o.step(dt)
        assert o.flags == 0
        compare(s.get_state(), o, FIELDS_2D, what="%s step %d" % (what, k), sigma_floor=1e-12)
        n_gpu = s.stats()["fallbacks"]
        assert n_gpu == o.fallbacks - before, (what, k, n_gpu, o.fallbacks - before)
        total += n_gpu
    s.close()
    return total


@pytest.mark.parametrize("order", [5, 9])
def test_double_mach_per_step(order):
    """48 x 12 cells on [0,4] x [0,1] (ragged tiles), 6 steps: inflow left,
    the split wall below, the moving shock split above."""
    nx, ny = 48, 12
    st, kw = inputs.double_mach(nx, ny, order)
    total = per_step_timed(order, nx, ny, st, kw, 6, "double Mach")
    assert total > 0  # the fallback was exercised


def test_oblique_shock_per_step_at_a_later_time():
    """The Mach 10 shock between four inflow sides, started at t = 0.004 so
    that the splits sit where the shock has moved (the state is the shock
    translated to that time)."""
    nx, ny, t0 = 24, 12, 0.004
    xa = 0.3
    st, kw = inputs.oblique_shock(nx, ny, 7, xa=xa + inputs.SHOCK_SPEED_X * t0)
    # splits of the shock started at xa, at time t0: the same positions
    kw["bc_split"][2:, 0] -= inputs.SHOCK_SPEED_X * t0
    o_kw = dict(tau_mode=cgks.TAU_HGKS, cfl=0.5, pt_fallback=1, **kw)
    o = oracle.Oracle(2, 7, nx, ny, **o_kw)
    o.set_state(*st)
    o.t = t0
    s = cgks.Solver(2, 7, nx, ny, **o_kw)
    for k in range(4):
        g0 = o.get_state()
        s.set_state(g0["W"], g0["Wx"], g0["Wy"], g0["Wx_line"], g0["Wy_line"], g0["sigma_x"], g0["sigma_y"])
        s.set_time(o.t)
        dt = o.compute_dt()
        before = o.fallbacks
        s.step(dt)
        s.sync()
        o.step(dt)
        assert o.flags == 0
        compare(s.get_state(), o, FIELDS_2D, what="oblique shock step %d" % k, sigma_floor=1e-12)
        assert s.stats()["fallbacks"] == o.fallbacks - before
    s.close()


def test_resume_with_initialised_sigma_takes_inflow_states_at_t0():
    """set_state without sigma, then set_time(t0): sigma is initialised again
    from the cell averages and the inflow ghost states at t0, as the oracle
    does for a state set at t0 (the moving splits have crossed a ghost cell
    by then, so the sigma of t = 0 differs); the next step matches too."""
    nx, ny, t0 = 24, 12, 0.004
    xa = 0.3
    st, kw = inputs.oblique_shock(nx, ny, 7, xa=xa + inputs.SHOCK_SPEED_X * t0)
    kw["bc_split"][2:, 0] -= inputs.SHOCK_SPEED_X * t0
    o_kw = dict(tau_mode=cgks.TAU_HGKS, cfl=0.5, pt_fallback=1, **kw)
    o0 = oracle.Oracle(2, 7, nx, ny, **o_kw)
    o0.set_state(*st)
    o = oracle.Oracle(2, 7, nx, ny, **o_kw)
    o.t = t0
    o.set_state(*st)
    assert not np.array_equal(o0.sx, o.sx) or not np.array_equal(o0.sy, o.sy)
    s = cgks.Solver(2, 7, nx, ny, **o_kw)
    s.set_state(*st)
    s.set_time(t0)
    g = s.get_state()
    assert np.allclose(g["sigma_x"], o.sx, rtol=1e-13, atol=1e-14)
    assert np.allclose(g["sigma_y"], o.sy, rtol=1e-13, atol=1e-14)
    dt = o.compute_dt()
    s.step(dt)
    s.sync()
    o.step(dt)
    compare(s.get_state(), o, FIELDS_2D, what="resumed oblique shock", sigma_floor=1e-12)
    s.close()


def test_fallback_off_reports_the_failure():
    """Without the fallback the first step of the double Mach reflection meets
    non-physical face states on the GPU as on the oracle, and says so."""
    nx, ny = 48, 12
    st, kw = inputs.double_mach(nx, ny, 5)
    s = cgks.Solver(2, 5, nx, ny, tau_mode=cgks.TAU_HGKS, cfl=0.5, **kw)
    s.set_state(*st)
    s.step(0.0)
    with pytest.raises(cgks.CgksError) as e:
        s.sync()
    assert e.value.code == cgks.ENONPHYS
    s.close()


def _top_row_front(rho, nx, x_end=4.0):
    """x where the top row's density first falls through 4.7 coming from the right."""
    r = rho[-1]
    k = int(np.nonzero(r > 4.7)[0][-1])
    h = x_end / nx
    return (k + 0.5 + (r[k] - 4.7) / (r[k] - r[k + 1])) * h


@pytest.mark.parametrize("prec", [cgks.FP32_BULK, cgks.FP64])
def test_double_mach_reflection_960x240(prec):
    """The paper's mesh, order 9, CFL 0.5, to t = 0.2: the run completes
    with every state positive, the fallback used, and the incident shock in
    the top row within two cells of its exact position
    1/6 + (y + 20 t) / sqrt 3 at the row's centre."""
    nx, ny, order, t_end = 960, 240, 9, 0.2
    st, kw = inputs.double_mach(nx, ny, order)
    s = cgks.Solver(2, order, nx, ny, precision=prec, tau_mode=cgks.TAU_HGKS, cfl=0.5, pt_fallback=1, **kw)
    s.set_state(*st)
    t, steps, code = s.run_to(t_end, max_steps=4000)
    W = s.get_state()["W"]
    fb = s.stats()["fallbacks"]
    s.close()
    assert code == 0 and t >= t_end - 1e-12, (code, t, steps)
    assert W[0].min() > 0 and _pressure(W).min() > 0
    assert fb > 0
    y_top = 1.0 - 0.5 / ny
    x_exact = 1.0 / 6.0 + (y_top + 20.0 * t_end) / np.sqrt(3.0)
    assert abs(_top_row_front(W[0], nx) - x_exact) < 2.0 * 4.0 / nx
