"""Parity at the benchmark's full size, in the launch configuration bench.py
times (one 2048^2 mesh, the CUDA-graph step with a device CFL time step).

The scheme is local: after one step a cell depends only on cells within 10
(two stages, each reaching 5 cells through Steps 1-3 and the DFF stencils).
So the oracle can compute sampled outputs exactly: it runs the same step on a
40 x 40 crop of the initial state around each sample, and the crop's inner
16 x 16 cells must equal the full-mesh GPU result."""
import numpy as np
import pytest

import oracle
from paper_2508_13705_gb300 import cgks, inputs

pytestmark = pytest.mark.gpu

CROP, MARGIN = 40, 12


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2508_13705_gb300 import build
    build.build()
    oracle.build()


def crop(a, j0, i0):
    """Periodic crop of the last two axes."""
    ny, nx = a.shape[-2:]
    jj = (np.arange(j0, j0 + CROP) % ny)[:, None]
    ii = (np.arange(i0, i0 + CROP) % nx)[None, :]
    return np.ascontiguousarray(a[..., jj, ii])


def sampled_oracle(st, ext_full, n, order, dt, centres, **kw):
    h = (ext_full[1] - ext_full[0]) / n
    out = []
    for (jc, ic) in centres:
        j0, i0 = jc - CROP // 2, ic - CROP // 2
        c = [crop(a, j0, i0) for a in st]
        o = oracle.Oracle(2, order, CROP, CROP, extent=(0.0, CROP * h, 0.0, CROP * h),
                          bc=(oracle.BC_TRANSMISSIVE,) * 4, **kw)
        o.set_state(*c)
        o.step(dt)
        out.append((j0, i0, o.get_state()))
    return out


def check(gpu_state, samples, tol, h, fields=("W", "Wx_line", "Wy_line")):
    """Cell averages: relative L1 <= tol.  Slopes: the same plus the rounding
    floor of differences of interface states over the cell size h (64 ulp of
    the largest state magnitude per value, as in test_gpu_parity)."""
    sl = slice(MARGIN, CROP - MARGIN)
    for j0, i0, o in samples:
        for f in fields:
            g = crop(gpu_state[f], j0, i0)[..., sl, sl]
            r = o[f][..., sl, sl]
            d = np.abs(g - r).sum()
            floor = 0.0 if f == "W" else r.size * 64 * np.finfo(float).eps * np.abs(o["W"]).max() / h
            assert d <= tol * np.abs(r).sum() + floor, (f, j0, i0, d / np.abs(r).sum())


def test_vortex_2048_order9_sampled_parity_fp64_and_fp32():
    n, order = 2048, 9
    ext = (0.0, 10.0, 0.0, 10.0)
    st = inputs.cell_state_2d(inputs.vortex_prim(), n, n, ext, order, nq=4)
    centres = [(1024, 1024), (700, 1300), (5, 2040)]  # the core, the flank, across the periodic corner
    results = {}
    for prec in (cgks.FP64, cgks.FP32_BULK):
        s = cgks.Solver(2, order, n, n, extent=ext, precision=prec)
        s.set_state(*st)
        dt = s.compute_dt()
        s.advance(1, 0.0)  # the bench's graph step: device CFL time step
        t, rc, _ = s.sync()
        assert rc == 0 and abs(t - dt) < 1e-15
        results[prec] = (dt, s.get_state())
        if prec == cgks.FP64:
            m0 = st[0].sum(axis=(1, 2))
            m1 = results[prec][1]["W"].sum(axis=(1, 2))
            assert np.all(np.abs(m1 - m0) <= 1e-12 * np.abs(m0))  # periodic: conserved
        s.close()
    dt = results[cgks.FP64][0]
    samples = sampled_oracle(st, ext, n, order, dt, centres)
    check(results[cgks.FP64][1], samples, 1e-12, 10.0 / n)
    check(results[cgks.FP32_BULK][1], samples, 1e-6, 10.0 / n, fields=("W",))


def test_vortex_1024_order9_autotuned_sampled_parity():
    """The bench's headline workload and launch shapes: 1024^2, autotuned
    (tile shapes and block sizes), one graph step with the device CFL step."""
    n, order = 1024, 9
    ext = (0.0, 10.0, 0.0, 10.0)
    st = inputs.vortex_2d(n, order)
    results = {}
    for prec in (cgks.FP64, cgks.FP32_BULK):
        s = cgks.Solver(2, order, n, n, extent=ext, precision=prec)
        s.set_state(*st)
        s.autotune()
        dt = s.compute_dt()
        s.advance(1, 0.0)
        t, rc, _ = s.sync()
        assert rc == 0 and abs(t - dt) < 1e-15
        results[prec] = (dt, s.get_state())
        s.close()
    dt = results[cgks.FP64][0]
    samples = sampled_oracle(st, ext, n, order, dt, [(512, 512), (300, 700), (3, 1020)])
    check(results[cgks.FP64][1], samples, 1e-12, 10.0 / n)
    check(results[cgks.FP32_BULK][1], samples, 1e-6, 10.0 / n, fields=("W",))


def test_quadrants_4096_order9_fp32_sampled():
    """Config C4 at full size (4096^2, FP32 bulk, transmissive, HGKS tau):
    two graph steps; samples near the quadrant corner and on a shock line."""
    n, order = 4096, 9
    st = inputs.quadrants_2d(n, order, seed=0)
    kw = dict(tau_mode=cgks.TAU_HGKS, bc=(cgks.BC_TRANSMISSIVE,) * 4)
    s = cgks.Solver(2, order, n, n, extent=(0.0, 1.0, 0.0, 1.0), precision=cgks.FP32_BULK, **kw)
    s.set_state(*st)
    dt = s.compute_dt()
    s.advance(1, dt)
    t, rc, _ = s.sync()
    assert rc == 0
    g = s.get_state()
    stats = s.stats()
    s.close()
    assert stats["min_rho"] > 0 and stats["min_p"] > 0
    samples = sampled_oracle(st, (0.0, 1.0, 0.0, 1.0), n, order, dt, [(2048, 2048), (1000, 2048), (2048, 3000)],
                             tau_mode=oracle.TAU_HGKS)
    check(g, samples, 2e-6, 1.0 / n, fields=("W",))
