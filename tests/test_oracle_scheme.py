"""Whole-scheme pins of the oracle: the paper's printed accuracy tables,
invariants the physics forces, and the exact Riemann solution."""
import os

import numpy as np
import pytest

import exact_riemann as er
from oracle import BC_TRANSMISSIVE, DFF_LAG_STAGE, DFF_LAG_STEP, TAU_HGKS, Oracle
from paper_2508_13705_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "accuracy_tables.txt")


def _table():
    t = {}
    for line in open(GOLD):
        if line.strip() and not line.startswith("#"):
            d, o, n, l1, l2, li = line.split()
            t[(int(d), int(o), int(n))] = (float(l1), float(l2), float(li))
    return t


TABLE = _table()


def run_wave(dim, order, N, **kw):
    dx = 2.0 / N
    dt = 0.3 * dx ** (order / 4)
    if dim == 1:
        o = Oracle(1, order, N, extent=(0, 2, 0, 1), **kw)
        o.set_state(*inputs.density_wave_1d(N))
        o.run(2.0, dt_fn=lambda s: dt)
        e = np.abs(o.W[0, 0] - inputs.density_wave_1d_exact_avg(N, 2.0))
    else:
        o = Oracle(2, order, N, N, extent=(0, 2, 0, 2), **kw)
        o.set_state(*inputs.density_wave_2d(N, order))
        o.run(2.0, dt_fn=lambda s: dt)
        e = np.abs(o.W[0] - inputs.density_wave_2d_exact_avg(N, 2.0))
    assert o.flags == 0
    return np.array([e.mean(), np.sqrt((e ** 2).mean()), e.max()])


# (dim, order, N, relative tolerance).  Orders 5 and 7 in 2-D and order 7 in
# 1-D reproduce all printed digits; 1-D order 5 and order 9 agree to a few
# per cent (the residual is not explained by the paper).
CASES = [(1, 7, 5, 2e-6), (1, 7, 10, 2e-6), (1, 7, 20, 2e-6),
         (2, 5, 5, 2e-6), (2, 5, 10, 2e-6), (2, 7, 5, 2e-6), (2, 7, 10, 2e-6),
         (1, 5, 10, 0.05), (1, 5, 20, 0.05), (1, 9, 10, 0.1), (1, 9, 20, 0.1),
         (2, 9, 5, 0.1), (2, 9, 10, 0.12)]


@pytest.mark.parametrize("dim,order,N,tol", CASES)
def test_printed_accuracy_tables(dim, order, N, tol):
    got = run_wave(dim, order, N)
    want = np.array(TABLE[(dim, order, N)])
    assert np.all(np.abs(got / want - 1) <= tol), (got, want)


@pytest.mark.parametrize("order", [5, 7, 9])
def test_design_order_1d(order):
    Ns = {5: (20, 40), 7: (10, 20), 9: (10, 20)}[order]
    e = [run_wave(1, order, N)[0] for N in Ns]
    assert abs(np.log2(e[0] / e[1]) - order) < 0.15


def test_riemann_configuration_3_all_orders_stay_positive():
    """Sec. 4.7 Configuration 3 (the paper's timing workload) on a coarse mesh:
    every order runs with CFL 0.5 and keeps rho, p > 0 (checked at every Gauss
    point by the oracle) over the first 0.15 time units."""
    n = 30
    S = np.array([[0.138, 1.206, 1.206, 0.029], [0.5323, 0, 1.206, 0.3], [1.5, 0, 0, 1.5],
                  [0.5323, 1.206, 0, 0.3]])
    xc = (np.arange(n) + 0.5) / n
    east = (xc >= 0.7)[None, :]
    north = (xc >= 0.7)[:, None]
    pr = S[np.where(north, np.where(east, 2, 3), np.where(east, 1, 0))]
    W = np.stack([pr[..., 0], pr[..., 0] * pr[..., 1], pr[..., 0] * pr[..., 2],
                  pr[..., 3] / 0.4 + 0.5 * pr[..., 0] * (pr[..., 1] ** 2 + pr[..., 2] ** 2)])
    for order in (5, 9):
        m = {5: 2, 9: 4}[order]
        z = np.zeros((4, n, n))
        o = Oracle(2, order, n, n, extent=(0, 1, 0, 1), tau_mode=TAU_HGKS, bc=(1, 1, 1, 1))
        o.set_state(W, z, z, np.zeros((m, 4, n, n)), np.zeros((m, 4, n, n)))
        o.run(0.15)
        assert o.flags == 0 and np.isfinite(o.W).all()


def test_order9_stable_at_cfl_half():
    """The paper runs every order at CFL 0.5.  With the Step 3 fit of degree
    min(3m-1, 8) the 2-D order-9 scheme is stable there (a degree-11
    interpolant through all 12 face points is not)."""
    N = 16
    o = Oracle(2, 9, N, N, extent=(0, 2, 0, 2), cfl=0.5)
    o.set_state(*inputs.density_wave_2d(N, 9))
    o.run(1.0)
    e = np.abs(o.W[0] - inputs.density_wave_2d_exact_avg(N, o.t)).mean()
    assert o.flags == 0 and e < 1e-4
    o = Oracle(2, 9, N, N, extent=(0, 2, 0, 2), cfl=0.5)
    o.P.step3_deg = 11
    o.set_state(*inputs.density_wave_2d(N, 9))
    o.run(1.0)
    assert o.flags != 0 or not np.isfinite(o.W).all()


def test_step3_literal_three_point_reading_misses_table():
    """Step 3 read as a 3-point difference at spacing dy gives third order in
    2-D, far from the printed 2-D table; the 3m-point Lagrange reading matches."""
    got = run_wave(2, 5, 10, step3=1)[0]
    assert got / TABLE[(2, 5, 10)][0] > 5


def test_flux_with_quadratic_term_is_second_order_in_time():
    """With the t^2/2 a_tt term kept in the flux integral, the linear flux fit of
    Eq. 2.19-2.20 leaves an O(dt^3) local error: the 1-D order-5 test converges
    at 2 x 5/4 = 2.5 and misses the printed table by orders of magnitude."""
    e = [run_wave(1, 5, N, )[0] for N in (20, 40)]
    o = []
    for N in (20, 40):
        dx = 2.0 / N
        s = Oracle(1, 5, N, extent=(0, 2, 0, 1))
        s.P.flux_tt = 1
        s.set_state(*inputs.density_wave_1d(N))
        s.run(2.0, dt_fn=lambda _: 0.3 * dx ** 1.25)
        o.append(np.abs(s.W[0, 0] - inputs.density_wave_1d_exact_avg(N, 2.0)).mean())
    assert abs(np.log2(o[0] / o[1]) - 2.5) < 0.2
    assert o[1] > 50 * e[1]


def test_free_stream_preservation():
    n = 12
    W = np.zeros((4, n, n))
    W[0], W[1], W[2] = 1.0, 0.3, -0.7
    W[3] = 1.0 / 0.4 + 0.5 * (0.09 + 0.49)
    for order in (5, 9):
        m = {5: 2, 9: 4}[order]
        o = Oracle(2, order, n, n, extent=(0, 1, 0, 1), tau_mode=TAU_HGKS)
        z = np.zeros((4, n, n))
        o.set_state(W, z, z, np.zeros((m, 4, n, n)), np.zeros((m, 4, n, n)))
        for _ in range(4):
            o.step()
        assert np.abs(o.W - W).max() <= 1e-14 * 3
        assert np.abs(o.Wx).max() <= 1e-12 and np.abs(o.Wyl).max() <= 1e-12


def test_conservation_periodic_with_shocks():
    n = 24
    st = inputs.quadrants_2d(n, 7, seed=0)
    o = Oracle(2, 7, n, n, extent=(0, 1, 0, 1), tau_mode=TAU_HGKS)
    o.set_state(*st)
    m0 = o.W.sum(axis=(1, 2))
    for _ in range(8):
        o.step()
    assert o.flags == 0
    assert np.all(np.abs(o.W.sum(axis=(1, 2)) - m0) <= 1e-13 * np.abs(m0).max() * n * n / 10)


def test_mirror_symmetry_1d():
    """A mirror-symmetric blast stays symmetric: checks the stencil orientation,
    the right-state mirroring and the AO linear weights."""
    n = 64
    x = (np.arange(n) + 0.5) / n
    rho = np.where(np.abs(x - 0.5) < 0.15, 2.0, 1.0)
    p = np.where(np.abs(x - 0.5) < 0.15, 5.0, 1.0)
    W = np.stack([rho, 0 * x, p / 0.4]).reshape(3, 1, n)
    for order in (5, 9):
        o = Oracle(1, order, n, extent=(0, 1, 0, 1), tau_mode=TAU_HGKS, bc=(1, 1, 1, 1))
        o.set_state(W, np.zeros_like(W))
        used_ao = False
        for _ in range(30):
            o.step()
            used_ao |= bool((o.branch == 0).any())
        assert used_ao  # the HWENO-AO branch was exercised
        w = o.W[:, 0]
        assert np.abs(w[0] - w[0, ::-1]).max() <= 1e-12
        assert np.abs(w[2] - w[2, ::-1]).max() <= 1e-12
        assert np.abs(w[1] + w[1, ::-1]).max() <= 1e-12


def test_rotation_symmetry_2d():
    """Transposing a 2-D problem (x <-> y, U <-> V) transposes the result."""
    n = 10
    st = inputs.quadrants_2d(n, 7, seed=3)
    W, Wx, Wy, Wxl, Wyl = st
    o1 = Oracle(2, 7, n, n, extent=(0, 1, 0, 1), tau_mode=TAU_HGKS, bc=(1, 1, 1, 1))
    o1.set_state(*st)
    T = lambda a: np.ascontiguousarray(np.swapaxes(a, -1, -2))
    Wt = T(W)[[0, 2, 1, 3]]
    o2 = Oracle(2, 7, n, n, extent=(0, 1, 0, 1), tau_mode=TAU_HGKS, bc=(1, 1, 1, 1))
    o2.set_state(np.ascontiguousarray(Wt), T(Wy)[[0, 2, 1, 3]], T(Wx)[[0, 2, 1, 3]],
                 T(Wyl)[:, [0, 2, 1, 3]], T(Wxl)[:, [0, 2, 1, 3]])
    for _ in range(3):
        o1.step(2e-3)
        o2.step(2e-3)
    assert np.abs(T(o1.W)[[0, 2, 1, 3]] - o2.W).max() <= 1e-13


def test_one_dimensional_flow_through_2d_scheme():
    """A flow uniform in y run by the 2-D scheme equals the 1-D scheme."""
    N = 16
    o1 = Oracle(1, 7, N, extent=(0, 2, 0, 1))
    o1.set_state(*inputs.density_wave_1d(N))
    f = lambda x, y: (1 + 0.2 * np.sin(np.pi * x), 1 + 0 * x, 0 * x, 1 + 0 * x)
    o2 = Oracle(2, 7, N, 2, extent=(0, 2, 0, 0.25))
    o2.set_state(*inputs.cell_state_2d(f, N, 2, (0, 2, 0, 0.25), 7))
    for _ in range(5):
        o1.step(0.01)
        o2.step(0.01)
    assert np.abs(o1.W[0, 0] - o2.W[0, 0]).max() <= 1e-13
    assert np.abs(o1.W[2, 0] - o2.W[3, 0]).max() <= 1e-13


@pytest.mark.parametrize("order", [5, 9])
def test_sod_against_exact_riemann(order):
    errs = []
    for N in (100, 200):
        o = Oracle(1, order, N, extent=(0, 1, 0, 1), tau_mode=TAU_HGKS, bc=(1, 1, 1, 1))
        o.set_state(*inputs.riemann_1d(N, *inputs.SOD))
        o.run(0.2)
        assert o.flags == 0 and o.W[0].min() > 0
        errs.append(np.abs(o.W[0, 0] - er.cell_average_rho(*inputs.SOD, N, 0.2)).mean())
    assert errs[0] < 5e-3 and errs[1] < 0.65 * errs[0]


def test_lax_positivity_and_error():
    N = 100
    o = Oracle(1, 9, N, extent=(0, 1, 0, 1), tau_mode=TAU_HGKS, bc=(1, 1, 1, 1))
    o.set_state(*inputs.riemann_1d(N, *inputs.LAX))
    o.run(0.14)
    assert o.flags == 0
    assert np.abs(o.W[0, 0] - er.cell_average_rho(*inputs.LAX, N, 0.14)).mean() < 2e-2


DOUBLE_RAREFACTION = ((1.0, -2.0, 0.1), (1.0, 2.0, 0.1))
LE_BLANC = ((1.0, 0.0, 2.0 / 3.0 * 1e-1), (1e-3, 0.0, 2.0 / 3.0 * 1e-10))


@pytest.mark.parametrize("order", [5, 9])
def test_double_rarefaction_against_exact_vacuum_solution(order):
    """Sec. 4.5: two rarefactions that leave a vacuum between them.  The
    scheme stays positive (min rho about 1e-6) and its L1 density error
    against the exact solution (two fans and a vacuum) falls with N."""
    errs = []
    for N in (100, 200):
        o = Oracle(1, order, N, extent=(0, 1, 0, 1), tau_mode=TAU_HGKS, bc=(1, 1, 1, 1))
        o.set_state(*inputs.riemann_1d(N, *DOUBLE_RAREFACTION))
        o.run(0.1)
        assert o.flags == 0 and o.W[0].min() > 0
        errs.append(np.abs(o.W[0, 0] - er.cell_average_rho(*DOUBLE_RAREFACTION, N, 0.1)).mean())
    assert errs[0] < 1.2e-2 and errs[1] < 0.7 * errs[0]


def test_le_blanc_loses_positivity_under_these_readings():
    """Sec. 4.5, Le Blanc (gamma = 5/3, N = 800, pressure ratio 1e9).  The
    paper reports a pass; under the readings of this build the first step
    leaves the cell next to the jump with a tiny positive pressure, and the
    second step meets a non-positive pressure at a face point, which the
    status flags report.  The kinetic flux with tau of the order of the step
    is not positivity-preserving at this ratio, and the paper states no
    limiter or first-step rule."""
    N, g = 800, 5.0 / 3.0
    o = Oracle(1, 5, N, extent=(0, 9, 0, 1), tau_mode=TAU_HGKS, bc=(1, 1, 1, 1), gamma=g)
    o.set_state(*inputs.riemann_1d(N, *LE_BLANC, x0=0.0, x1=9.0, xs=3.0, gamma=g))
    o.step(o.compute_dt())
    assert o.flags == 0 and o.W[0].min() > 0
    o.step(o.compute_dt())
    assert o.flags != 0


STRONG_TUBE = ((120.0, 0.0, 120.0 / 1.4), (1.2, 0.0, 1.2 / 1.4))  # the initial jump of Sec. 4.9


def test_stage_lag_reading_carries_a_strong_shock_tube():
    """Sec. 3.1 takes sigma "from the previous time step".  With the step lag a
    strong wave (density and pressure ratio 100, the jump of Sec. 4.9) crosses
    into cells whose stencils still see sigma = 0 in stage 2 of step 2: a
    linear stencil spans the huge slope of the shocked cell and a face point
    turns negative.  With sigma of stage 1 of the same step in stage 2 the
    tube runs, and its density error against the exact solution falls with N."""
    o = Oracle(1, 9, 100, extent=(0, 1, 0, 1), tau_mode=TAU_HGKS, bc=(1, 1, 1, 1), cfl=0.2,
               dff_lag=DFF_LAG_STEP)
    o.set_state(*inputs.riemann_1d(100, *STRONG_TUBE))
    o.step(o.compute_dt())
    o.step(o.compute_dt())
    assert o.flags != 0
    errs = []
    for N in (100, 200):
        o = Oracle(1, 9, N, extent=(0, 1, 0, 1), tau_mode=TAU_HGKS, bc=(1, 1, 1, 1), cfl=0.2,
                   dff_lag=DFF_LAG_STAGE)
        o.set_state(*inputs.riemann_1d(N, *STRONG_TUBE))
        o.run(0.1)
        assert o.flags == 0 and o.W[0].min() > 0
        errs.append(np.abs(o.W[0, 0] - er.cell_average_rho(*STRONG_TUBE, N, 0.1)).mean())
    assert errs[1] < 0.7 * errs[0]


def test_stage_lag_equals_step_lag_on_smooth_data():
    """Smooth data keep every sigma far below the threshold, so both readings
    take the same branches and give the same result to the last bit."""
    res = []
    for lag in (DFF_LAG_STEP, DFF_LAG_STAGE):
        o = Oracle(1, 7, 40, extent=(0, 2, 0, 1), dff_lag=lag)
        o.set_state(*inputs.density_wave_1d(40))
        for _ in range(20):
            o.step(2e-3)
        res.append(o.W.copy())
    assert np.array_equal(res[0], res[1])


def _blast(N=400, cfl=0.5, **kw):
    g = 1.4
    o = Oracle(1, 5, N, extent=(0, 1, 0, 1), tau_mode=TAU_HGKS, bc=(3, 3, 1, 1), gamma=g, cfl=cfl, **kw)
    x = (np.arange(N) + 0.5) / N
    p = np.where(x < 0.1, 1000.0, np.where(x > 0.9, 100.0, 0.01))
    W = np.zeros((3, 1, N))
    W[0] = 1.0
    W[2] = p / (g - 1)
    o.set_state(W, np.zeros((3, 1, N)))
    return o


@pytest.mark.parametrize("cfl,positive", [(0.5, False), (0.2, False), (0.05, True)])
def test_blast_wave_first_step_loses_positivity_ahead_of_the_jump(cfl, positive):
    """Sec. 4.4, Woodward-Colella (pressure ratio 1e5, reflective walls, 400
    cells).  The paper reports a pass at CFL 0.5; under the readings of this
    build the first step leaves the second low-pressure cell (cell 41, one
    face ahead of the jump) with a negative pressure: in stage 2 the wave has
    reached its left face, and the S2O4 combination weights that face's flux
    only through the stage-2 time derivative F_t*, which a flux switching on
    within the step does not represent.  A smaller step (CFL 0.05) keeps the
    first step positive.  The same holds with the DFF time lag of stage 2,
    with the collision time taken from the two cells' pressures, with the
    literal flux integral and with larger c1 or c2 (the design notes list
    them); none is a reading that passes."""
    o = _blast(cfl=cfl)
    o.step(o.compute_dt())
    W = o.W[:, 0]
    p = 0.4 * (W[2] - 0.5 * W[1] ** 2 / W[0])
    assert (p.min() > 0) == positive
    if not positive:
        assert int(p.argmin()) == 41
