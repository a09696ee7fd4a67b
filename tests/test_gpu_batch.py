"""Batched persistent stepping of uneven meshes (config C5 shape).

A batch advances all instances with one persistent launch per kernel inside
one CUDA graph per step.  Every instance must agree with the same instance
run alone through the single-mesh entry points to rounding: a single mesh
runs a separate compilation of the stage kernels (its descriptor passed by
value), which may contract multiply-adds differently.  The FP64 batch must
match the oracle."""
import numpy as np
import pytest

import oracle
from paper_2508_13705_gb300 import cgks, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2508_13705_gb300 import build
    build.build()
    oracle.build()


def specs(n=5, seed=3):
    return inputs.batch_specs(n, seed=seed, lo=12, hi=40)


def ext_of(sp):
    return (0.0, 1.0, 0.0, sp["ny"] / sp["nx"])


@pytest.mark.parametrize("precision,kw", [
    (cgks.FP64, {}), (cgks.FP32_BULK, {}),
    # slip walls and the viscous collision time: the wall instances of the
    # stencil kernels and the viscous flux inside the batch graph
    (cgks.FP64, dict(bc=(cgks.BC_REFLECTIVE, cgks.BC_REFLECTIVE, cgks.BC_NOSLIP, cgks.BC_NOSLIP),
                     tau_mode=cgks.TAU_NS, mu=1e-3))])
def test_batch_equals_single_instances(precision, kw):
    sp = specs()
    order = 7
    states = [inputs.batch_instance(s, order) for s in sp]
    kw = dict(dict(tau_mode=cgks.TAU_HGKS), **kw)
    b = cgks.Batch(order, [s["nx"] for s in sp], [s["ny"] for s in sp], [ext_of(s) for s in sp],
                   precision=precision, **kw)
    for k, st in enumerate(states):
        b.set_state(k, *st)
    dts = np.array([2e-4 * (1 + 0.1 * k) for k in range(len(sp))])
    for _ in range(3):
        b.step(dts)
    b.step(None)  # a CFL step: every instance takes its own time step
    b.sync()
    for k, (s, st) in enumerate(zip(sp, states)):
        one = cgks.Solver(2, order, s["nx"], s["ny"], extent=ext_of(s), precision=precision, **kw)
        one.set_state(*st)
        for _ in range(3):
            one.step(dts[k])
        one.step(0.0)
        one.sync()
        g1, gb = one.get_state(), b.get_state(k)
        # FP64: rounding-level; FP32 bulk: the parity bounds of its increments
        l1_tol, max_tol = (1e-12, 1e-10) if precision == cgks.FP64 else (5e-8, 5e-6)
        for f in ("W", "Wx", "Wy", "Wx_line", "Wy_line"):
            d, ref = np.abs(g1[f] - gb[f]), np.abs(g1[f])
            assert d.sum() <= l1_tol * ref.sum(), (k, f, d.sum() / ref.sum())
            assert d.max() <= max_tol * ref.max(), (k, f, d.max() / ref.max())


def test_batch_instance_matches_oracle():
    sp = specs(3, seed=5)
    order = 7
    states = [inputs.batch_instance(s, order) for s in sp]
    b = cgks.Batch(order, [s["nx"] for s in sp], [s["ny"] for s in sp], [ext_of(s) for s in sp],
                   tau_mode=cgks.TAU_HGKS)
    for k, st in enumerate(states):
        b.set_state(k, *st)
    dts = np.full(len(sp), 3e-4)
    for _ in range(2):
        b.step(dts)
    b.sync()
    for k, (s, st) in enumerate(zip(sp, states)):
        o = oracle.Oracle(2, order, s["nx"], s["ny"], extent=ext_of(s), tau_mode=oracle.TAU_HGKS)
        o.set_state(*st)
        o.step(3e-4)
        o.step(3e-4)
        g = b.get_state(k)
        assert np.abs(g["W"] - o.W).sum() / np.abs(o.W).sum() <= 1e-12, k
        # slopes: the same bound plus the rounding floor of differences of
        # interface states over the cell size (see test_gpu_parity.slope_floor)
        floor = 64 * np.finfo(float).eps * np.abs(o.W).max() / min(o.dx, o.dy)
        for f, ref in (("Wx_line", o.Wxl), ("Wy_line", o.Wyl)):
            d = np.abs(g[f] - ref).sum()
            assert d <= 1e-12 * np.abs(ref).sum() + ref.size * floor, (k, f, d)


def test_batch_with_degenerate_instances_matches_oracle():
    """Instances smaller than a stencil (1 x 1, 2 x 3, 5 x 1) beside an
    ordinary one in one batch: the descriptor table, the work lists and the
    periodic wrap of each, against the oracle per instance."""
    order = 9
    dims = [(1, 1), (2, 3), (5, 1), (17, 9)]

    def prim(x, y):
        return 1 + 0.2 * np.sin(2 * np.pi * (x + 2 * y)), 0.5 + 0 * x, -0.3 + 0 * x, 1 + 0 * x
    ext = (0.0, 1.0, 0.0, 1.0)
    states = [inputs.cell_state_2d(prim, nx, ny, ext, order) for nx, ny in dims]
    b = cgks.Batch(order, [d[0] for d in dims], [d[1] for d in dims], [ext] * len(dims))
    for k, st in enumerate(states):
        b.set_state(k, *st)
    dts = np.array([1e-3 * (1 + 0.5 * k) for k in range(len(dims))])
    for _ in range(2):
        b.step(dts)
    b.sync()
    for k, ((nx, ny), st) in enumerate(zip(dims, states)):
        o = oracle.Oracle(2, order, nx, ny, extent=ext)
        o.set_state(*st)
        o.step(dts[k])
        o.step(dts[k])
        g = b.get_state(k)
        assert np.abs(g["W"] - o.W).sum() <= 1e-12 * np.abs(o.W).sum(), k
        floor = 64 * np.finfo(float).eps * np.abs(o.W).max() / min(o.dx, o.dy)
        for f, ref in (("Wx_line", o.Wxl), ("Wy_line", o.Wyl)):
            d = np.abs(g[f] - ref).sum()
            assert d <= 1e-12 * np.abs(ref).sum() + ref.size * floor, (k, f, d)


def test_batch_device_state_calls_equal_host_calls():
    """cgks_batch_set_state_device / _get_state_device (CUDA tensors, enqueued
    on the batch's stream) give bitwise the same steps as the host-array calls,
    in both precision forms."""
    import torch
    sp = specs(4, seed=9)
    order = 5
    states = [inputs.batch_instance(s, order) for s in sp]
    names = ("W", "Wx", "Wy", "Wx_line", "Wy_line")
    for precision in (cgks.FP64, cgks.FP32_BULK):
        args = ([s["nx"] for s in sp], [s["ny"] for s in sp], [ext_of(s) for s in sp])
        bh = cgks.Batch(order, *args, precision=precision, tau_mode=cgks.TAU_HGKS)
        bd = cgks.Batch(order, *args, precision=precision, tau_mode=cgks.TAU_HGKS,
                        stream=torch.cuda.current_stream().cuda_stream)
        for k, st in enumerate(states):
            bh.set_state(k, *st)
            bd.set_state_device(k, *[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in st])
        for _ in range(2):
            bh.step(None)
            bd.step(None)
        bh.sync()
        bd.sync()
        for k, st in enumerate(states):
            out = {n: torch.empty(a.shape, dtype=torch.float64, device="cuda") for n, a in zip(names, st)}
            bd.get_state_device(k, out)
            torch.cuda.synchronize()
            gh = bh.get_state(k)
            for n in names:
                assert np.array_equal(out[n].cpu().numpy(), gh[n]), (precision, k, n)
        bh.close()
        bd.close()
