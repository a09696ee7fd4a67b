"""ctypes binding of the C ABI in include/cgks.h (argument marshalling only).

Every step of the scheme runs in the CUDA kernels of ``_build/libcgks.so``;
this module only converts arrays and parameters.  If the library has not been
built the binding raises: there is no CPU fallback.

Host arrays are float64 numpy arrays in the layouts of the C ABI:
W, Wx, Wy ``[nvar][ny][nx]``, Wx_line / Wy_line ``[m][nvar][ny][nx]``,
sigma_x ``[ny][nx+1]``, sigma_y ``[ny+1][nx]``.  Device arrays may be given as
CUDA torch tensors (float64, contiguous) to the ``*_device`` calls.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcgks.so")

FP64, FP32_BULK = 0, 1
TAU_ZERO, TAU_HGKS, TAU_NS = 0, 1, 2
DFF_LAG_STEP, DFF_LAG_STAGE = 0, 1
BC_PERIODIC, BC_TRANSMISSIVE, BC_FIXED, BC_REFLECTIVE, BC_NOSLIP = 0, 1, 2, 3, 4
BC_INFLOW, BC_INFLOW_REFLECTIVE = 5, 6
PT_FALLBACK_OFF, PT_FALLBACK_FIRST_ORDER = 0, 1
EINVAL, ENOMEM, ECUDA, ENONPHYS, ETIMEOUT, ENOTSUP = -1, -2, -3, -4, -5, -6

EXPORTS = ("cgks_default_params", "cgks_init_mesh", "cgks_set_state", "cgks_set_state_device",
           "cgks_set_ghost", "cgks_compute_dt", "cgks_step", "cgks_advance", "cgks_sync",
           "cgks_get_state", "cgks_get_state_device", "cgks_get_stats", "cgks_step_info",
           "cgks_destroy", "cgks_strerror", "cgks_batch_init", "cgks_batch_set_state",
           "cgks_batch_step", "cgks_batch_sync", "cgks_batch_get_state", "cgks_batch_destroy",
           "cgks_stencil_row", "cgks_profile_step", "cgks_step_1d_noalloc", "cgks_autotune",
           "cgks_batch_autotune", "cgks_set_time", "cgks_batch_set_state_device",
           "cgks_batch_get_state_device", "cgks_fma_peak")


class Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("order", ctypes.c_int), ("precision", ctypes.c_int),
                ("tau_mode", ctypes.c_int), ("bc", ctypes.c_int * 4), ("gamma", ctypes.c_double),
                ("cfl", ctypes.c_double), ("sigma_thres", ctypes.c_double), ("gamma_hi", ctypes.c_double),
                ("gamma_lo", ctypes.c_double), ("weno_eps", ctypes.c_double), ("tau_c1", ctypes.c_double),
                ("tau_c2", ctypes.c_double), ("mu", ctypes.c_double), ("dff_lag", ctypes.c_int),
                ("pt_fallback", ctypes.c_int), ("bc_state", ctypes.c_double * 32),
                ("bc_split", ctypes.c_double * 8)]


class Stats(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("steps", ctypes.c_longlong), ("min_rho", ctypes.c_double),
                ("min_p", ctypes.c_double), ("mass", ctypes.c_double * 4), ("branch", ctypes.c_longlong * 4),
                ("fallbacks", ctypes.c_longlong)]


class CgksError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed: %s (%d)" % (what, strerror(code), code))
        self.code = code


_lib = None


def lib():
    """Load libcgks.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libcgks.so is not built (%s); run paper_2508_13705_gb300.build.build()"
                               % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
        L.cgks_default_params.argtypes = [ctypes.POINTER(Params), ip, ip]
        L.cgks_init_mesh.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Params), ip, ip, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, vp]
        L.cgks_set_state.argtypes = [vp] + [vp] * 7
        L.cgks_set_state_device.argtypes = [vp] + [vp] * 7
        L.cgks_set_ghost.argtypes = [vp, vp]
        L.cgks_compute_dt.argtypes = [vp, dp]
        L.cgks_step.argtypes = [vp, ctypes.c_double]
        L.cgks_set_time.argtypes = [vp, ctypes.c_double]
        L.cgks_advance.argtypes = [vp, ip, ctypes.c_double]
        L.cgks_sync.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_longlong)]
        L.cgks_get_state.argtypes = [vp] + [vp] * 7
        L.cgks_get_state_device.argtypes = [vp] + [vp] * 7
        L.cgks_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        L.cgks_step_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        L.cgks_destroy.argtypes = [vp]
        L.cgks_destroy.restype = None
        L.cgks_strerror.argtypes = [ip]
        L.cgks_strerror.restype = ctypes.c_char_p
        L.cgks_batch_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Params), ip, vp, vp, vp, vp]
        L.cgks_batch_set_state.argtypes = [vp, ip] + [vp] * 5
        L.cgks_batch_step.argtypes = [vp, vp]
        L.cgks_batch_sync.argtypes = [vp]
        L.cgks_batch_get_state.argtypes = [vp, ip] + [vp] * 5
        L.cgks_batch_set_state_device.argtypes = [vp, ip] + [vp] * 5
        L.cgks_batch_get_state_device.argtypes = [vp, ip] + [vp] * 5
        L.cgks_batch_destroy.argtypes = [vp]
        L.cgks_batch_destroy.restype = None
        L.cgks_stencil_row.argtypes = [ip, ip, ip, dp]
        L.cgks_profile_step.argtypes = [vp, ctypes.c_double, ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.cgks_autotune.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        L.cgks_batch_autotune.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        L.cgks_fma_peak.argtypes = [ip, dp, ctypes.POINTER(ctypes.c_float)]
        L.cgks_step_1d_noalloc.argtypes = [ctypes.POINTER(Params), ip, ctypes.c_double, ctypes.c_double,
                                           vp, vp, vp, vp, ctypes.c_double, vp, vp]
        _lib = L
    return _lib


def strerror(code):
    return lib().cgks_strerror(code).decode()


def _check(code, what):
    if code != 0:
        raise CgksError(code, what)


def _host(a, shape=None):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.size != int(np.prod(shape)):
        raise ValueError("array of %d values where %s was expected" % (a.size, shape))
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _dev(t):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()):
        raise ValueError("device arrays must be contiguous float64 CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


TUNED_KEYS = ("recon_x", "recon_y", "flux1", "flux2", "update1", "update2", "tile_x", "tile_y")


def _tuned(fn, h):
    t = (ctypes.c_int * 10)()
    _check(fn(h, t), "autotune")
    v = list(t)
    return dict(zip(TUNED_KEYS, v[:6] + [(v[6], v[7]), (v[8], v[9])]))


def make_params(dim, order, precision=FP64, tau_mode=TAU_ZERO, bc=(BC_PERIODIC,) * 4, **kw):
    p = Params()
    _check(lib().cgks_default_params(ctypes.byref(p), dim, order), "cgks_default_params")
    p.precision, p.tau_mode = precision, tau_mode
    for k in range(4):
        p.bc[k] = bc[k]
    for k, v in kw.items():
        if k in ("bc_state", "bc_split"):
            # [4][2][4] inflow states and [4][2] split points, flattened in C order
            v = np.asarray(v, dtype=np.float64).ravel().tolist()
            getattr(p, k)[:] = v
        else:
            setattr(p, k, v)
    return p


class Solver:
    """One mesh.  ``stream``: a cudaStream_t value (int) or None (own stream)."""

    def __init__(self, dim, order, nx, ny=1, extent=(0.0, 1.0, 0.0, 1.0), precision=FP64,
                 tau_mode=TAU_ZERO, bc=(BC_PERIODIC,) * 4, stream=None, **kw):
        self.dim, self.order, self.nx = dim, order, nx
        self.ny = ny if dim == 2 else 1
        self.nv = dim + 2
        self.m = {5: 2, 7: 3, 9: 4}[order] if dim == 2 else 1
        self.params = make_params(dim, order, precision, tau_mode, bc, **kw)
        h = ctypes.c_void_p()
        x0, x1, y0, y1 = extent
        _check(lib().cgks_init_mesh(ctypes.byref(h), ctypes.byref(self.params), nx, self.ny, x0, x1, y0, y1,
                                    ctypes.c_void_p(stream or 0)), "cgks_init_mesh")
        self.h = h

    # shapes
    def _shapes(self):
        c = (self.nv, self.ny, self.nx)
        return dict(W=c, Wx=c, Wy=c, Wx_line=(self.m,) + c, Wy_line=(self.m,) + c,
                    sigma_x=(self.ny, self.nx + 1), sigma_y=(self.ny + 1, self.nx))

    def set_state(self, W, Wx, Wy=None, Wx_line=None, Wy_line=None, sigma_x=None, sigma_y=None):
        sh = self._shapes()
        keep, ptrs = [], []
        for name, a in (("W", W), ("Wx", Wx), ("Wy", Wy), ("Wx_line", Wx_line), ("Wy_line", Wy_line),
                        ("sigma_x", sigma_x), ("sigma_y", sigma_y)):
            if self.dim == 1 and name in ("Wy", "Wx_line", "Wy_line", "sigma_y"):
                a = None
            arr, p = _host(a, sh[name])
            keep.append(arr)
            ptrs.append(p)
        _check(lib().cgks_set_state(self.h, *ptrs), "cgks_set_state")

    def set_state_device(self, W, Wx, Wy=None, Wx_line=None, Wy_line=None, sigma_x=None, sigma_y=None):
        _check(lib().cgks_set_state_device(self.h, *[_dev(t) for t in (W, Wx, Wy, Wx_line, Wy_line,
                                                                         sigma_x, sigma_y)]),
               "cgks_set_state_device")

    def set_ghost(self, ghost):
        arr, p = _host(ghost, (36,))
        _check(lib().cgks_set_ghost(self.h, p), "cgks_set_ghost")

    def get_state(self, out=None):
        """Copy the state to the host as FP64 arrays (dict keyed W, Wx, ...).
        ``out``: optional dict of caller-owned C-contiguous float64 arrays of
        the right sizes (pinned ones give the fastest copies), filled in place
        and returned."""
        sh = self._shapes()
        names = ["W", "Wx", "Wy", "Wx_line", "Wy_line", "sigma_x", "sigma_y"]
        if self.dim == 1:
            names = ["W", "Wx", "sigma_x"]
        if out is None:
            out = {n: np.zeros(sh[n]) for n in names}
        else:
            for n in names:
                a = out[n]
                if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
                        and a.size == int(np.prod(sh[n]))):
                    raise ValueError("out[%r] must be a C-contiguous float64 array of %s values" % (n, sh[n]))
        ptr = lambda n: out[n].ctypes.data_as(ctypes.c_void_p) if n in out else None
        _check(lib().cgks_get_state(self.h, *[ptr(n) for n in ("W", "Wx", "Wy", "Wx_line", "Wy_line",
                                                                 "sigma_x", "sigma_y")]), "cgks_get_state")
        return out

    def get_state_device(self, out):
        """Copy the state into preallocated CUDA tensors (dict keyed like get_state)."""
        _check(lib().cgks_get_state_device(self.h, *[_dev(out.get(n)) for n in (
            "W", "Wx", "Wy", "Wx_line", "Wy_line", "sigma_x", "sigma_y")]), "cgks_get_state_device")

    def compute_dt(self):
        d = ctypes.c_double()
        _check(lib().cgks_compute_dt(self.h, ctypes.byref(d)), "cgks_compute_dt")
        return d.value

    def step(self, dt=0.0):
        _check(lib().cgks_step(self.h, float(dt)), "cgks_step")

    def run_to(self, t_end, t=0.0, max_steps=10 ** 6, check_every=64):
        """Advance from time ``t`` to ``t_end`` with the CFL step, the last step
        clipped.  Returns (t, steps, status).  Stops early when the device
        status reports a non-physical state (checked every ``check_every``
        steps and whenever the CFL step stops being positive and finite: a
        blown-up state gives a vanishing step that would never reach t_end) or
        after ``max_steps``."""
        steps = 0
        while t < t_end - 1e-14 * max(1.0, abs(t_end)) and steps < max_steps:
            dt = self.compute_dt()
            if not (dt > 1e-14 * max(1.0, abs(t_end))) or dt != dt or steps % check_every == check_every - 1:
                _, code, _ = self.sync(raise_on_error=False)
                if code or not (dt > 1e-14 * max(1.0, abs(t_end))):
                    return t, steps, code or ENONPHYS
            dt = min(dt, t_end - t)
            self.step(dt)
            t += dt
            steps += 1
        _, code, _ = self.sync(raise_on_error=False)
        return t, steps, code

    def advance(self, n, dt=0.0):
        _check(lib().cgks_advance(self.h, int(n), float(dt)), "cgks_advance")

    def sync(self, raise_on_error=True):
        t = ctypes.c_double()
        bad = ctypes.c_longlong()
        r = lib().cgks_sync(self.h, ctypes.byref(t), ctypes.byref(bad))
        if r and raise_on_error:
            raise CgksError(r, "cgks_sync (first flagged index %d)" % bad.value)
        return t.value, r, bad.value

    def stats(self):
        s = Stats()
        _check(lib().cgks_get_stats(self.h, ctypes.byref(s)), "cgks_get_stats")
        return dict(t=s.t, min_rho=s.min_rho, min_p=s.min_p, mass=list(s.mass)[: self.nv],
                    branch=dict(zip(("ao", "r5", "r7", "r9"), list(s.branch))), fallbacks=s.fallbacks)

    def set_time(self, t):
        """Set the simulated time t^n of the next step (restarts, inflow split points)."""
        _check(lib().cgks_set_time(self.h, float(t)), "cgks_set_time")

    def autotune(self):
        """Pick each stage kernel's launch shape by timing it on the current state."""
        return _tuned(lib().cgks_autotune, self.h)

    def kernels_per_step(self):
        n = ctypes.c_int()
        _check(lib().cgks_step_info(self.h, ctypes.byref(n)), "cgks_step_info")
        return n.value

    def profile_step(self, dt):
        """One fixed-dt step kernel by kernel: list of (kernel id, device ms)."""
        ms = (ctypes.c_float * 16)()
        ids = (ctypes.c_int * 16)()
        n = ctypes.c_int(16)
        _check(lib().cgks_profile_step(self.h, float(dt), ms, ids, ctypes.byref(n)), "cgks_profile_step")
        return [(ids[k], ms[k]) for k in range(n.value)]

    def close(self):
        if getattr(self, "h", None):
            lib().cgks_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent 2-D meshes stepped by shared persistent launches."""

    def __init__(self, order, nx, ny, extents, precision=FP64, tau_mode=TAU_ZERO, bc=(BC_PERIODIC,) * 4,
                 stream=None, **kw):
        self.order, self.n = order, len(nx)
        self.nx, self.ny = list(nx), list(ny)
        self.m = {5: 2, 7: 3, 9: 4}[order]
        self.params = make_params(2, order, precision, tau_mode, bc, **kw)
        self._nx = np.ascontiguousarray(nx, dtype=np.int32)
        self._ny = np.ascontiguousarray(ny, dtype=np.int32)
        self._ext = np.ascontiguousarray(extents, dtype=np.float64).reshape(-1)
        h = ctypes.c_void_p()
        _check(lib().cgks_batch_init(ctypes.byref(h), ctypes.byref(self.params), self.n,
                                     self._nx.ctypes.data_as(ctypes.c_void_p),
                                     self._ny.ctypes.data_as(ctypes.c_void_p),
                                     self._ext.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(stream or 0)),
               "cgks_batch_init")
        self.h = h

    def set_state(self, k, W, Wx, Wy, Wx_line, Wy_line):
        c = (4, self.ny[k], self.nx[k])
        arrs = [_host(W, c), _host(Wx, c), _host(Wy, c), _host(Wx_line, (self.m,) + c),
                _host(Wy_line, (self.m,) + c)]
        _check(lib().cgks_batch_set_state(self.h, k, *[a[1] for a in arrs]), "cgks_batch_set_state")

    def set_state_device(self, k, W, Wx, Wy, Wx_line, Wy_line):
        """Instance k from float64 CUDA tensors, enqueued on the batch's stream."""
        _check(lib().cgks_batch_set_state_device(self.h, k, *[_dev(t) for t in (W, Wx, Wy, Wx_line, Wy_line)]),
               "cgks_batch_set_state_device")

    def get_state_device(self, k, out):
        """Instance k into preallocated float64 CUDA tensors (dict keyed W, Wx, Wy, Wx_line, Wy_line)."""
        _check(lib().cgks_batch_get_state_device(self.h, k, *[_dev(out.get(n)) for n in (
            "W", "Wx", "Wy", "Wx_line", "Wy_line")]), "cgks_batch_get_state_device")

    def step(self, dt=None):
        if dt is None:
            _check(lib().cgks_batch_step(self.h, None), "cgks_batch_step")
        else:
            d = np.ascontiguousarray(dt, dtype=np.float64)
            _check(lib().cgks_batch_step(self.h, d.ctypes.data_as(ctypes.c_void_p)), "cgks_batch_step")

    def sync(self):
        _check(lib().cgks_batch_sync(self.h), "cgks_batch_sync")

    def autotune(self):
        return _tuned(lib().cgks_batch_autotune, self.h)

    def get_state(self, k):
        c = (4, self.ny[k], self.nx[k])
        out = dict(W=np.zeros(c), Wx=np.zeros(c), Wy=np.zeros(c), Wx_line=np.zeros((self.m,) + c),
                   Wy_line=np.zeros((self.m,) + c))
        _check(lib().cgks_batch_get_state(self.h, k, *[out[n].ctypes.data_as(ctypes.c_void_p) for n in (
            "W", "Wx", "Wy", "Wx_line", "Wy_line")]), "cgks_batch_get_state")
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().cgks_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fma_peak(precision):
    """Measured FMA throughput of the current GPU (TFLOP/s) in FP32 or FP64."""
    t = ctypes.c_double()
    ms = ctypes.c_float()
    _check(lib().cgks_fma_peak(precision, ctypes.byref(t), ctypes.byref(ms)), "cgks_fma_peak")
    return t.value, ms.value


def stencil_row(order, st, row):
    out = (ctypes.c_double * 10)()
    _check(lib().cgks_stencil_row(order, st, row, out), "cgks_stencil_row")
    return np.array(out[:])
