"""1-D robustness suite on the GPU (Sec. 4.2 and 4.5): the Lax shock tube, the
double rarefaction that leaves a near-vacuum, and the Le Blanc problem.

Parity with the FP64 oracle is checked per step from the same state (the DFF
branches near the waves must agree exactly), and whole GPU runs are checked
against the exact Riemann solution with the oracle's own error as the bar.
"""
import numpy as np
import pytest

import exact_riemann as er
import oracle
from paper_2508_13705_gb300 import cgks, inputs
from test_gpu_parity import FIELDS_1D, compare

pytestmark = pytest.mark.gpu

DOUBLE_RAREFACTION = ((1.0, -2.0, 0.1), (1.0, 2.0, 0.1))
LE_BLANC = ((1.0, 0.0, 2.0 / 3.0 * 1e-1), (1e-3, 0.0, 2.0 / 3.0 * 1e-10))
HG = dict(tau_mode=cgks.TAU_HGKS, bc=(1, 1, 1, 1))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2508_13705_gb300 import build
    build.build()
    oracle.build()


def mach2(states, gamma):
    """Largest squared Mach number of the initial states."""
    return max(u * u * rho / (gamma * p) for rho, u, p in states)


def per_step(order, N, st, steps, extent=(0, 1, 0, 1), gamma=1.4, what="", ma2=1.0):
    """Per-step parity from the oracle's state.  The sigma rounding floor of
    Eq. 3.2 scales with the squared Mach numbers it differences."""
    floor = 1e-14 * max(1.0, ma2)
    o = oracle.Oracle(1, order, N, extent=extent, gamma=gamma, **HG)
    o.set_state(*st)
    s = cgks.Solver(1, order, N, extent=extent, gamma=gamma, **HG)
    branches = set()
    for k in range(steps):
        g0 = o.get_state()
        s.set_state(g0["W"], g0["Wx"], sigma_x=g0["sigma_x"])
        dt = o.compute_dt()
        s.step(dt)
        s.sync()
        o.step(dt)
        branches |= set(np.unique(o.branch).tolist())
        compare(s.get_state(), o, FIELDS_1D, what="%s step %d" % (what, k), sigma_floor=floor)
    s.close()
    return branches


@pytest.mark.parametrize("order", [5, 7, 9])
def test_double_rarefaction_per_step(order):
    """The paper's mesh (N = 400): 30 steps, through the formation of the
    near-vacuum, with the HWENO-AO branch active at the fan edges."""
    st = inputs.riemann_1d(400, *DOUBLE_RAREFACTION)
    branches = per_step(order, 400, st, 30, what="double rarefaction", ma2=mach2(DOUBLE_RAREFACTION, 1.4))
    assert 0 in branches  # HWENO-AO used


@pytest.mark.parametrize("order", [7, 9])
def test_lax_per_step(order):
    st = inputs.riemann_1d(100, *inputs.LAX)
    branches = per_step(order, 100, st, 25, what="Lax", ma2=mach2(inputs.LAX, 1.4))
    assert 0 in branches


def gpu_run(order, N, st, t_end, extent=(0, 1, 0, 1), gamma=1.4):
    """GPU alone to t_end with the CFL step (the last step clipped)."""
    s = cgks.Solver(1, order, N, extent=extent, gamma=gamma, **HG)
    s.set_state(*st)
    t, steps, code = s.run_to(t_end, max_steps=20000)
    assert code == 0 and t >= t_end - 1e-12, (code, t, steps)
    out = s.get_state()
    s.close()
    return out


@pytest.mark.parametrize("order", [5, 9])
def test_double_rarefaction_full_run_against_exact(order):
    """To t = 0.1 at N = 400 on the GPU: positive throughout, and the L1
    density error against the exact vacuum solution equals the oracle's
    (same steps, FP64) to 1e-9 relative."""
    N = 400
    st = inputs.riemann_1d(N, *DOUBLE_RAREFACTION)
    g = gpu_run(order, N, st, 0.1)
    o = oracle.Oracle(1, order, N, extent=(0, 1, 0, 1), **HG)
    o.set_state(*st)
    o.run(0.1)
    exact = er.cell_average_rho(*DOUBLE_RAREFACTION, N, 0.1)
    e_gpu = np.abs(g["W"][0, 0] - exact).mean()
    e_orc = np.abs(o.W[0, 0] - exact).mean()
    assert g["W"][0].min() > 0
    assert e_gpu < 5e-3
    assert abs(e_gpu - e_orc) <= 1e-9 * e_orc


def test_lax_full_run_against_exact():
    N = 100
    st = inputs.riemann_1d(N, *inputs.LAX)
    g = gpu_run(9, N, st, 0.14)
    e = np.abs(g["W"][0, 0] - er.cell_average_rho(*inputs.LAX, N, 0.14)).mean()
    assert e < 2e-2


def test_le_blanc_first_step_matches_and_loss_is_reported():
    """Le Blanc (gamma = 5/3, N = 800): the first step matches the oracle;
    the second meets a non-positive pressure at a face point under this
    build's readings (the oracle flags the same step), and the device status
    reports it through cgks_sync as CGKS_ENONPHYS without a fault."""
    N, gam = 800, 5.0 / 3.0
    ext = (0, 9, 0, 1)
    st = inputs.riemann_1d(N, *LE_BLANC, x0=0.0, x1=9.0, xs=3.0, gamma=gam)
    per_step(5, N, st, 1, extent=ext, gamma=gam, what="Le Blanc", ma2=mach2(LE_BLANC, gam))
    o = oracle.Oracle(1, 5, N, extent=ext, gamma=gam, **HG)
    o.set_state(*st)
    s = cgks.Solver(1, 5, N, extent=ext, gamma=gam, **HG)
    s.set_state(*st)
    for k in range(2):
        dt = o.compute_dt()
        o.step(dt)
        s.step(dt)
    assert o.flags != 0
    _, code, bad = s.sync(raise_on_error=False)
    assert code == cgks.ENONPHYS and bad >= 0
    s.close()
