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
