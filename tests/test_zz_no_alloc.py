"""The 1-D step that allocates no device memory, against the solver path.

Some callers cannot call cudaMalloc: code that runs under another
framework's memory manager, which owns the device, or code on a path where an
allocation (and the device synchronisation it may imply) is not allowed.
``cgks_step_1d_noalloc`` serves them with a fixed scratch array inside the
library.  This test calls it twice in a row through the C ABI (the second
call starts from the first call's output) and compares each result with the
same steps taken by the ordinary solver entry points.
"""
import ctypes

import numpy as np
import pytest

from paper_2508_13705_gb300 import build, cgks, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


def test_noalloc_step_matches_solver_on_two_calls():
    import torch
    build.build()
    L = cgks.lib()
    N, order = 400, 9
    W, Wx = inputs.riemann_1d(N, *inputs.SOD)
    kw = dict(tau_mode=cgks.TAU_HGKS, bc=(cgks.BC_TRANSMISSIVE,) * 4)
    s = cgks.Solver(1, order, N, extent=(0.0, 1.0, 0.0, 1.0), **kw)
    s.set_state(W, Wx)
    dt = s.compute_dt()
    ref = []
    for _ in range(2):
        s.step(dt)
        s.sync()
        ref.append(s.get_state())
    s.close()

    p = cgks.make_params(1, order, **kw)
    dev = torch.device("cuda")
    st0 = torch.from_numpy(np.concatenate([W.reshape(-1), Wx.reshape(-1)])).to(dev)
    st = [st0, torch.empty_like(st0), torch.empty_like(st0)]
    sg = [None, torch.empty(N + 1, dtype=torch.float64, device=dev), torch.empty(N + 1, dtype=torch.float64, device=dev)]
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    stream = torch.cuda.current_stream().cuda_stream
    free_before = None
    for k in range(2):
        rc = L.cgks_step_1d_noalloc(ctypes.byref(p), N, 0.0, 1.0, ptr(st[k]), ptr(sg[k]), ptr(st[k + 1]),
                                    ptr(sg[k + 1]), dt, ptr(status), ctypes.c_void_p(stream))
        assert rc == 0, cgks.strerror(rc)
        torch.cuda.synchronize()
        if k == 0:
            free_before = torch.cuda.mem_get_info()[0]
        out = st[k + 1].cpu().numpy()
        assert int(status.item()) == 0
        assert rel_l1(out[: 3 * N], ref[k]["W"].reshape(-1)) <= TOL
        assert rel_l1(out[3 * N:], ref[k]["Wx"].reshape(-1)) <= TOL
        sig = sg[k + 1].cpu().numpy()
        assert np.all(np.abs(sig - ref[k]["sigma_x"].reshape(-1)) <= TOL * np.abs(ref[k]["sigma_x"].reshape(-1)) + 1e-14)
    # the second call took no device memory
    assert torch.cuda.mem_get_info()[0] == free_before


def _noalloc_two_calls(L, p, N, W, Wx, dts):
    """Two chained no-allocation steps from (W, Wx); returns the two states."""
    import torch
    dev = torch.device("cuda")
    st0 = torch.from_numpy(np.concatenate([W.reshape(-1), Wx.reshape(-1)])).to(dev)
    st = [st0, torch.empty_like(st0), torch.empty_like(st0)]
    sg = [None, torch.empty(N + 1, dtype=torch.float64, device=dev), torch.empty(N + 1, dtype=torch.float64, device=dev)]
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for k in range(2):
        rc = L.cgks_step_1d_noalloc(ctypes.byref(p), N, 0.0, 1.0, ptr(st[k]), ptr(sg[k]), ptr(st[k + 1]),
                                    ptr(sg[k + 1]), dts[k], ptr(status), ctypes.c_void_p(stream))
        assert rc == 0, cgks.strerror(rc)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        outs.append((st[k + 1].cpu().numpy().copy(), sg[k + 1].cpu().numpy().copy()))
    return outs


@pytest.mark.parametrize("precision", [cgks.FP64, cgks.FP32_BULK])
def test_noalloc_cfl_step_matches_solver(precision):
    """dt <= 0 (the CFL step evaluated on the device inside the call) in both
    precision forms: the same kernels as the solver's CFL step, bitwise."""
    build.build()
    L = cgks.lib()
    N, order = 256, 7
    W, Wx = inputs.riemann_1d(N, *inputs.SOD)
    kw = dict(tau_mode=cgks.TAU_HGKS, bc=(cgks.BC_TRANSMISSIVE,) * 4, precision=precision)
    s = cgks.Solver(1, order, N, extent=(0.0, 1.0, 0.0, 1.0), **kw)
    s.set_state(W, Wx)
    ref = []
    for _ in range(2):
        s.step(0.0)
        s.sync()
        ref.append(s.get_state())
    s.close()
    outs = _noalloc_two_calls(L, cgks.make_params(1, order, **kw), N, W, Wx, (0.0, 0.0))
    for (out, sig), r in zip(outs, ref):
        assert np.array_equal(out[: 3 * N], r["W"].reshape(-1))
        assert np.array_equal(out[3 * N:], r["Wx"].reshape(-1))
        assert np.array_equal(sig, r["sigma_x"].reshape(-1))


def test_noalloc_step_matches_oracle():
    """FP64 no-allocation steps against the FP64 CPU oracle on the same
    seeded shock tube (relative L1 within 1e-12 per field, and the largest
    single deviation within 1e-10 of the field's scale)."""
    import oracle
    oracle.build()
    build.build()
    L = cgks.lib()
    N, order = 200, 9
    W, Wx = inputs.riemann_1d(N, *inputs.SOD)
    kw = dict(tau_mode=cgks.TAU_HGKS, bc=(cgks.BC_TRANSMISSIVE,) * 4)
    o = oracle.Oracle(1, order, N, extent=(0.0, 1.0, 0.0, 1.0), tau_mode=oracle.TAU_HGKS,
                      bc=(oracle.BC_TRANSMISSIVE,) * 4)
    o.set_state(W, Wx)
    dts = (o.compute_dt(), 0.9 * o.compute_dt())
    outs = _noalloc_two_calls(L, cgks.make_params(1, order, **kw), N, W, Wx, dts)
    for (out, sig), dt in zip(outs, dts):
        o.step(dt)
        for got, want in ((out[: 3 * N], o.W.reshape(-1)), (out[3 * N:], o.Wx.reshape(-1))):
            assert rel_l1(got, want) <= TOL
            assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


def test_noalloc_rejects_oversized_and_unsupported():
    import torch
    L = cgks.lib()
    p = cgks.make_params(1, 5)
    buf = torch.zeros(6 * 5000, dtype=torch.float64, device="cuda")
    sig = torch.zeros(5001, dtype=torch.float64, device="cuda")
    a = ctypes.c_void_p(buf.data_ptr())
    b = ctypes.c_void_p(sig.data_ptr())
    assert L.cgks_step_1d_noalloc(ctypes.byref(p), 4097, 0.0, 1.0, a, None, a, b, 1e-3, None, None) == cgks.EINVAL
    p2 = cgks.make_params(2, 5)
    assert L.cgks_step_1d_noalloc(ctypes.byref(p2), 64, 0.0, 1.0, a, None, a, b, 1e-3, None, None) == cgks.EINVAL
    p3 = cgks.make_params(1, 5, bc=(cgks.BC_FIXED, 1, 1, 1))
    assert L.cgks_step_1d_noalloc(ctypes.byref(p3), 64, 0.0, 1.0, a, None, a, b, 1e-3, None, None) == cgks.ENOTSUP
