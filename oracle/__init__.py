"""FP64 CPU oracle of the ASE-DFF compact gas-kinetic scheme (S2O4 step).

TEST INFRASTRUCTURE ONLY.  This package is the independent, slow, plain
reference that the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may import it; the product path never does.  It shares no code,
header or table generator with the CUDA library.

Split of the work:

* ``cgks_oracle.c`` (plain C, FP64, loops in the paper's order) evaluates,
  for every face Gauss point of one stage, the time-integrated fluxes
  F(dt), F(dt/2) (Eq. 2.15) and the interface states W(0), W(dt/2), W(dt)
  (Eq. 2.11) after the reconstruction of Sec. 3 and the kinetic weighting of
  Eq. 2.7-2.8; and the discontinuity strength of Eq. 3.2 at each point.
* This module does the two-stage fourth-order time stepping exactly as
  Eq. 2.19-2.23 (fluxes) and Eq. 2.25, 2.29, 2.30 plus the Gauss-theorem slope
  update of Sec. 3.3 (cell and line slopes), in numpy.

Readings of the paper (each also listed in the design notes):

* DFF lag: sigma from the stage-1 left/right states of step n-1 feeds both
  stages of step n ("previous time step", Sec. 3.1).
* initial sigma: Eq. 3.2 applied to the two adjacent cell averages.
* Gauss weights normalised to sum 1 in every face sum (Sec. 3.3 prints the
  sums without weights).
"""
import ctypes
import os
import subprocess

import numpy as np

from . import coeffs

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

BC_PERIODIC, BC_TRANSMISSIVE, BC_FIXED, BC_REFLECTIVE, BC_NOSLIP = 0, 1, 2, 3, 4
BC_INFLOW, BC_INFLOW_REFLECTIVE = 5, 6
TAU_ZERO, TAU_HGKS, TAU_NS = 0, 1, 2
DFF_LAG_STEP, DFF_LAG_STAGE = 0, 1


def build(force=False):
    """Compile the C oracle (gcc, FP64, no FMA contraction)."""
    src = os.path.join(_HERE, "cgks_oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                           "-std=c11", "-D_DEFAULT_SOURCE", "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


_SO_COUNT = os.path.join(_BUILD, "liboracle_count.so")


def build_tally(force=False):
    """Compile the operation-counting build of the same C source (flopcount.cpp)."""
    srcs = [os.path.join(_HERE, "cgks_oracle.c"), os.path.join(_HERE, "flopcount.cpp")]
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO_COUNT) and all(
            os.path.getmtime(_SO_COUNT) >= os.path.getmtime(f) for f in srcs):
        return _SO_COUNT
    tmp = _SO_COUNT + ".tmp%d" % os.getpid()
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-w",
                           "-o", tmp, srcs[1]], cwd=_HERE)
    os.replace(tmp, _SO_COUNT)
    return _SO_COUNT


class OParams(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("order", ctypes.c_int), ("m", ctypes.c_int),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("bc", ctypes.c_int * 4),
                ("tau_mode", ctypes.c_int), ("step3", ctypes.c_int), ("flux_tt", ctypes.c_int),
                ("dff_faces", ctypes.c_int), ("step3_deg", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("gamma", ctypes.c_double),
                ("sigma_thres", ctypes.c_double), ("gamma_hi", ctypes.c_double),
                ("gamma_lo", ctypes.c_double), ("weno_eps", ctypes.c_double),
                ("c1", ctypes.c_double), ("c2", ctypes.c_double), ("mu", ctypes.c_double),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("tb", ctypes.c_double),
                ("bcs", ctypes.c_double * 32), ("bcx", ctypes.c_double * 8), ("pt_fallback", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(OParams)
        ip = ctypes.POINTER(ctypes.c_int)
        _lib.oracle_faces_1d.argtypes = [P, dp, dp, dp, dp, dp, ctypes.c_double, dp, dp, ip, ip]
        _lib.oracle_faces_2d.argtypes = [P, dp, dp, ctypes.c_int, dp, dp, dp, dp, dp, dp, dp,
                                         ctypes.c_double, dp, dp, ip]
        for f in ("oracle_point_1d", "oracle_point_2d"):
            getattr(_lib, f).argtypes = [P, dp, dp, ctypes.c_double, dp]
        _lib.oracle_moments.argtypes = [P, dp, dp, dp, dp]
        _lib.oracle_micro_slope.argtypes = [P, dp, dp, dp]
        _lib.oracle_recon.argtypes = [P, dp, dp, dp, dp]
        _lib.oracle_smoothness.argtypes = [dp, ctypes.c_int]
        _lib.oracle_smoothness.restype = ctypes.c_double
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def gauss_points(order):
    """m = 2, 3, 4 Gauss points per face for orders 5, 7, 9 (Sec. 3.3)."""
    return {5: 2, 7: 3, 9: 4}[order]


class Oracle:
    """Plain FP64 solver: state arrays in SoA layout, as the C-ABI uses.

    W, Wx, Wy: [nvar][ny][nx]; Wx_line, Wy_line: [m][nvar][ny][nx];
    sigma_x: [ny][nx+1]; sigma_y: [ny+1][nx].  1-D: ny = 1, nvar = 3.
    """

    def __init__(self, dim, order, nx, ny=1, extent=(0.0, 1.0, 0.0, 1.0), gamma=1.4, cfl=0.5,
                 tau_mode=TAU_ZERO, bc=(BC_PERIODIC,) * 4, sigma_thres=1.0, gamma_hi=0.85,
                 gamma_lo=0.6, weno_eps=1e-8, c1=0.05, c2=1.0, step3=0, mu=0.0, dff_lag=DFF_LAG_STEP,
                 bc_state=None, bc_split=None, pt_fallback=0):
        assert dim in (1, 2) and order in (5, 7, 9)
        assert dim == 2 or not any(b in (BC_INFLOW, BC_INFLOW_REFLECTIVE) for b in bc)
        self.dim, self.order, self.nx, self.ny = dim, order, nx, (ny if dim == 2 else 1)
        self.nv = dim + 2
        self.m = gauss_points(order) if dim == 2 else 1
        x0, x1, y0, y1 = extent
        self.dx = (x1 - x0) / nx
        self.dy = (y1 - y0) / self.ny if dim == 2 else 1.0
        self.gamma, self.cfl = gamma, cfl
        self.bc = tuple(bc)
        P = OParams()
        P.dim, P.order, P.m, P.nx, P.ny = dim, order, self.m, nx, self.ny
        for k in range(4):
            P.bc[k] = bc[k]
        P.tau_mode, P.step3 = tau_mode, step3
        # Step 3 fit: degree min(3m-1, 8) through the 3m face points of three segments
        P.step3_deg = min(3 * self.m - 1, 8) if dim == 2 else 0
        P.dx, P.dy, P.gamma = self.dx, self.dy, gamma
        P.sigma_thres, P.gamma_hi, P.gamma_lo = sigma_thres, gamma_hi, gamma_lo
        P.weno_eps, P.c1, P.c2 = weno_eps, c1, c2
        P.mu = mu
        # inflow sides: ghost cells hold bc_state[side][0] where the centre
        # coordinate along the side is below bc_split[side][0] + bc_split[side][1] t,
        # bc_state[side][1] beyond (conservative variables)
        self.x0, self.y0 = x0, y0
        self.bc_state = np.zeros((4, 2, 4)) if bc_state is None else np.asarray(bc_state, dtype=np.float64).reshape(4, 2, 4)
        self.bc_split = np.zeros((4, 2)) if bc_split is None else np.asarray(bc_split, dtype=np.float64).reshape(4, 2)
        P.x0, P.y0 = x0, y0
        P.bcs[:] = self.bc_state.ravel().tolist()
        P.bcx[:] = self.bc_split.ravel().tolist()
        # flagged option (the paper states no limiter): a face point side whose
        # reconstructed state is not physical falls back to its cell's average
        P.pt_fallback = pt_fallback
        self.fallbacks = 0
        self.mu, self.tau_mode = mu, tau_mode
        # reading of the DFF time lag (Sec. 3.1): sigma of stage 1 of step n-1
        # in both stages of step n (STEP), or in stage 2 the sigma of stage 1 of
        # the same step (STAGE)
        self.dff_lag = dff_lag
        self.P = P
        tabs = coeffs.poly_tables()
        self.T = np.ascontiguousarray(np.stack([tabs[k] for k in ("S0", "S1", "S2", "r5", "r7", "r9")]))
        gx, gw = coeffs.gauss_legendre_unit(self.m) if dim == 2 else (np.zeros(1), np.ones(1))
        self.gx, self.gw = np.ascontiguousarray(gx), np.ascontiguousarray(gw)
        self.ghost = None
        self.t = 0.0
        self.flags = 0
        self.branch = None

    # ---------------------------------------------------------------- state
    def set_state(self, W, Wx, Wy=None, Wx_line=None, Wy_line=None, sigma_x=None, sigma_y=None,
                  ghost=None):
        c = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64).copy()
        self.W, self.Wx, self.Wy = c(W), c(Wx), c(Wy)
        self.Wxl, self.Wyl = c(Wx_line), c(Wy_line)
        if ghost is not None:
            self.ghost = np.ascontiguousarray(ghost, dtype=np.float64).reshape(2, 3, 2, 3).copy()
        if self.dim == 1:
            self.Wy = self.Wxl = self.Wyl = None
        self.fallbacks = 0
        if sigma_x is None:
            sigma_x, sigma_y = self.initial_sigma()
        self.sx = c(sigma_x)
        self.sy = c(sigma_y) if self.dim == 2 else None

    def get_state(self):
        return dict(W=self.W.copy(), Wx=self.Wx.copy(),
                    Wy=None if self.Wy is None else self.Wy.copy(),
                    Wx_line=None if self.Wxl is None else self.Wxl.copy(),
                    Wy_line=None if self.Wyl is None else self.Wyl.copy(),
                    sigma_x=self.sx.copy(), sigma_y=None if self.sy is None else self.sy.copy())

    def _neighbour_states(self, axis):
        """Cell averages at both sides of every face along ``axis`` (ghost rule applied)."""
        W = self.W
        n = W.shape[2 - axis]
        lo_bc, hi_bc = self.bc[2 * axis], self.bc[2 * axis + 1]
        take = lambda k: np.take(W, [k], axis=2 - axis)

        def mirror(q, bc):
            # the wall's ghost cell: the adjacent cell with the normal momentum
            # (slip) or every momentum component (no-slip) reversed
            q = q.copy()
            for v in range(1, self.nv - 1):
                if v == 1 + axis or bc == BC_NOSLIP:
                    q[v] = -q[v]
            return q

        def prescribed(side, wall):
            # centres along the side against its split point at the current time
            if axis == 0:
                s = self.y0 + (np.arange(self.ny) + 0.5) * self.dy
                s = s.reshape(1, -1, 1)
            else:
                s = self.x0 + (np.arange(self.nx) + 0.5) * self.dx
                s = s.reshape(1, 1, -1)
            below = s < self.bc_split[side, 0] + self.bc_split[side, 1] * self.t
            a = self.bc_state[side, 0].reshape(-1, 1, 1)
            b = wall if wall is not None else self.bc_state[side, 1].reshape(-1, 1, 1)
            return np.where(below, a, b)

        if lo_bc == BC_PERIODIC:
            lo = take(n - 1)
        elif lo_bc == BC_FIXED:
            lo = self.ghost[0, 0, 0].reshape(-1, 1, 1)
        elif lo_bc in (BC_REFLECTIVE, BC_NOSLIP):
            lo = mirror(take(0), lo_bc)
        elif lo_bc in (BC_INFLOW, BC_INFLOW_REFLECTIVE):
            lo = prescribed(2 * axis, mirror(take(0), lo_bc) if lo_bc == BC_INFLOW_REFLECTIVE else None)
        else:
            lo = take(0)
        if hi_bc == BC_PERIODIC:
            hi = take(0)
        elif hi_bc == BC_FIXED:
            hi = self.ghost[1, 0, 0].reshape(-1, 1, 1)
        elif hi_bc in (BC_REFLECTIVE, BC_NOSLIP):
            hi = mirror(take(n - 1), hi_bc)
        elif hi_bc in (BC_INFLOW, BC_INFLOW_REFLECTIVE):
            hi = prescribed(2 * axis + 1, mirror(take(n - 1), hi_bc) if hi_bc == BC_INFLOW_REFLECTIVE else None)
        else:
            hi = take(n - 1)
        ext = np.concatenate([lo, W, hi], axis=2 - axis)
        sl = [slice(None)] * 3
        sl[2 - axis] = slice(0, n + 1)
        left = ext[tuple(sl)]
        sl[2 - axis] = slice(1, n + 2)
        right = ext[tuple(sl)]
        return left, right

    def _sigma_pair(self, Wl, Wr, axis):
        """Eq. 3.2 from two conservative states (normal velocity along ``axis``)."""
        g, dim = self.gamma, self.dim

        def prim(Wq):
            rho = Wq[0]
            u = Wq[1] / rho
            v = Wq[2] / rho if dim == 2 else 0.0 * rho
            p = (g - 1.0) * (Wq[dim + 1] - 0.5 * rho * (u * u + v * v))
            a = np.sqrt(g * p / rho)
            un, ut = (u, v) if axis == 0 else (v, u)
            return p, un / a, ut / a

        pl, mnl, mtl = prim(Wl)
        pr, mnr, mtr = prim(Wr)
        dp = np.abs(pl - pr)
        return dp / pl + dp / pr + (mnl - mnr) ** 2 + (mtl - mtr) ** 2

    def initial_sigma(self):
        """Reading: at t = 0 sigma comes from the two adjacent cell averages."""
        l, r = self._neighbour_states(0)
        sx = np.ascontiguousarray(self._sigma_pair(l, r, 0))
        if self.dim == 1:
            return sx, None
        l, r = self._neighbour_states(1)
        sy = np.ascontiguousarray(self._sigma_pair(l, r, 1))
        return sx, sy

    # ---------------------------------------------------------------- physics
    def compute_dt(self):
        """CFL rule (Sec. 4): dt = C * min over cells of h / (|U| + a_s), and for
        viscous flow also of h^2 / (4 nu) with nu = mu / rho."""
        W, g = self.W, self.gamma
        rho = W[0]
        u = W[1] / rho
        v = W[2] / rho if self.dim == 2 else 0.0
        p = (g - 1.0) * (W[self.dim + 1] - 0.5 * rho * (u * u + v * v))
        a = np.sqrt(g * p / rho)
        h = min(self.dx, self.dy) if self.dim == 2 else self.dx
        lim = h / (np.sqrt(u * u + v * v) + a)
        if self.tau_mode == TAU_NS and self.mu > 0:
            lim = np.minimum(lim, h * h / (4.0 * self.mu / rho))
        return float(self.cfl * np.min(lim))

    def faces(self, dt, state=None):
        """One stage's face evaluation.  Returns (out_x, sig_x[, out_y, sig_y])."""
        L = lib()
        W, Wx, Wy, Wxl, Wyl = state if state is not None else (self.W, self.Wx, self.Wy, self.Wxl, self.Wyl)
        nx, ny, m = self.nx, self.ny, self.m
        if self.dim == 1:
            out = np.zeros((5, 3, nx + 1))
            sig = np.zeros(nx + 1)
            br = np.zeros(nx + 2, dtype=np.int32)
            gh = self.ghost if self.ghost is not None else np.zeros((2, 3, 2, 3))
            nf = ctypes.c_int(0)
            fl = L.oracle_faces_1d(ctypes.byref(self.P), _p(self.T), _p(W), _p(Wx), _p(self.sx),
                                   _p(np.ascontiguousarray(gh)), dt, _p(out), _p(sig),
                                   br.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.byref(nf))
            self.flags |= fl
            self.fallbacks += nf.value
            self.branch = br
            return out.reshape(5, 3, 1, nx + 1), sig
        ox = np.zeros((5, 4, ny, nx + 1, m))
        sgx = np.zeros((ny, nx + 1, m))
        oy = np.zeros((5, 4, ny + 1, nx, m))
        sgy = np.zeros((ny + 1, nx, m))
        args = (_p(W), _p(Wx), _p(Wy), _p(Wxl), _p(Wyl), _p(self.sx), _p(self.sy), dt)
        for d, (o, sg) in enumerate(((ox, sgx), (oy, sgy))):
            nf = ctypes.c_int(0)
            self.flags |= L.oracle_faces_2d(ctypes.byref(self.P), _p(self.T), _p(self.gx), d, *args, _p(o), _p(sg),
                                            ctypes.byref(nf))
            self.fallbacks += nf.value
        return ox, sgx, oy, sgy

    # Gauss-weighted face differences of a face quantity q
    def _dfx(self, q):
        if self.dim == 1:
            return q[..., 1:] - q[..., :-1]
        return np.einsum("vjil,l->vji", q[:, :, 1:, :] - q[:, :, :-1, :], self.gw)

    def _dgy(self, q):
        return np.einsum("vjil,l->vji", q[:, 1:, :, :] - q[:, :-1, :, :], self.gw)

    def _lines_x(self, q):
        # [v][j][f][l] -> [l][v][j][i] line slopes (W_{i+1/2,l} - W_{i-1/2,l}) / dx
        d = (q[:, :, 1:, :] - q[:, :, :-1, :]) / self.dx
        return np.ascontiguousarray(np.transpose(d, (3, 0, 1, 2)))

    def _lines_y(self, q):
        d = (q[:, 1:, :, :] - q[:, :-1, :, :]) / self.dy
        return np.ascontiguousarray(np.transpose(d, (3, 0, 1, 2)))

    def step(self, dt=None):
        """One S2O4 step (Eq. 2.13, 2.19-2.25, 2.29-2.30)."""
        if dt is None or dt <= 0:
            dt = self.compute_dt()
        dx, dy = self.dx, self.dy
        W, Wx, Wy, Wxl, Wyl = self.W, self.Wx, self.Wy, self.Wxl, self.Wyl
        # ---- stage 1 at t^n
        self.P.tb = self.t
        r1 = self.faces(dt)
        ox = r1[0]
        Fd, Fh, W0, Wh, Wd = ox
        F1 = (4.0 * Fh - Fd) / dt                      # Eq. 2.19
        Ft1 = 4.0 * (Fd - 2.0 * Fh) / dt ** 2          # Eq. 2.20
        Wt1 = (4.0 * Wh - 3.0 * W0 - Wd) / dt          # Eq. 2.29
        Wtt1 = 4.0 * (Wd + W0 - 2.0 * Wh) / dt ** 2
        Ws = W - self._dfx(Fh) / dx                    # Eq. 2.21
        if self.dim == 2:
            oy = r1[2]
            Gd, Gh, V0, Vh, Vd = oy
            G1 = (4.0 * Gh - Gd) / dt
            Gt1 = 4.0 * (Gd - 2.0 * Gh) / dt ** 2
            Vt1 = (4.0 * Vh - 3.0 * V0 - Vd) / dt
            Vtt1 = 4.0 * (Vd + V0 - 2.0 * Vh) / dt ** 2
            Ws = Ws - self._dgy(Gh) / dy
            # f* = f(dt/2) (Eq. 2.26 with Eq. 2.28): slopes from W(dt/2)
            Wxls = self._lines_x(Wh)
            Wyls = self._lines_y(Vh)
            Wxs = np.einsum("lvji,l->vji", Wxls, self.gw)
            Wys = np.einsum("lvji,l->vji", Wyls, self.gw)
            sig_x_new = r1[1].mean(axis=2)             # Eq. 3.1
            sig_y_new = r1[3].mean(axis=2)
        else:
            Wxs = (Wh[..., 1:] - Wh[..., :-1]) / dx    # Eq. 2.30 at t*
            Wys = Wxls = Wyls = None
            sig_x_new = r1[1].reshape(1, -1)
        # ---- stage 2 at t* (same dt)
        if self.dff_lag == DFF_LAG_STAGE:
            self.sx = np.ascontiguousarray(sig_x_new)
            if self.dim == 2:
                self.sy = np.ascontiguousarray(sig_y_new)
        self.P.tb = self.t + 0.5 * dt
        r2 = self.faces(dt, state=(np.ascontiguousarray(Ws), np.ascontiguousarray(Wxs),
                                   None if Wys is None else np.ascontiguousarray(Wys), Wxls, Wyls))
        Fd2, Fh2, W02, Wh2, Wd2 = r2[0]
        Ft2 = 4.0 * (Fd2 - 2.0 * Fh2) / dt ** 2
        Wtt2 = 4.0 * (Wd2 + W02 - 2.0 * Wh2) / dt ** 2
        Fn = F1 + dt / 6.0 * (Ft1 + 2.0 * Ft2)         # Eq. 2.22
        Wf = W0 + dt * Wt1 + dt ** 2 / 6.0 * (Wtt1 + 2.0 * Wtt2)   # Eq. 2.25
        Wn = W - dt / dx * self._dfx(Fn)               # Eq. 2.23
        if self.dim == 2:
            Gd2, Gh2, V02, Vh2, Vd2 = r2[2]
            Gt2 = 4.0 * (Gd2 - 2.0 * Gh2) / dt ** 2
            Vtt2 = 4.0 * (Vd2 + V02 - 2.0 * Vh2) / dt ** 2
            Gn = G1 + dt / 6.0 * (Gt1 + 2.0 * Gt2)
            Vf = V0 + dt * Vt1 + dt ** 2 / 6.0 * (Vtt1 + 2.0 * Vtt2)
            Wn = Wn - dt / dy * self._dgy(Gn)
            self.Wxl = self._lines_x(Wf)
            self.Wyl = self._lines_y(Vf)
            self.Wx = np.ascontiguousarray(np.einsum("lvji,l->vji", self.Wxl, self.gw))
            self.Wy = np.ascontiguousarray(np.einsum("lvji,l->vji", self.Wyl, self.gw))
            self.sy = np.ascontiguousarray(sig_y_new)
        else:
            self.Wx = np.ascontiguousarray((Wf[..., 1:] - Wf[..., :-1]) / dx)
        self.W = np.ascontiguousarray(Wn)
        self.sx = np.ascontiguousarray(sig_x_new)
        self.t += dt
        return dt

    def run(self, t_end, dt_fn=None, max_steps=10 ** 7):
        """Advance to t_end; ``dt_fn(solver)`` overrides the CFL rule; last step clipped."""
        n = 0
        while self.t < t_end - 1e-14 * max(1.0, t_end) and n < max_steps:
            dt = dt_fn(self) if dt_fn else self.compute_dt()
            dt = min(dt, t_end - self.t)
            self.step(dt)
            n += 1
        return n

    # ---------------------------------------------------------------- single-point probes
    def point(self, Dl, Dr, dt):
        """Kinetic evaluation at one face point.  Dl, Dr: [3][nv] (1-D: W, W_x, W_xx)
        or [6][4] (2-D local frame: W, W_n, W_nn, W_t, W_tt, W_nt).
        Returns [5][nv]: F(dt), F(dt/2), W(0), W(dt/2), W(dt); and the flag."""
        nv = self.nv
        out = np.zeros((5, nv))
        f = lib().oracle_point_1d if self.dim == 1 else lib().oracle_point_2d
        fl = f(ctypes.byref(self.P), _p(np.ascontiguousarray(Dl, dtype=np.float64)),
               _p(np.ascontiguousarray(Dr, dtype=np.float64)), dt, _p(out))
        return out, fl

    def moments(self, W):
        mu = np.zeros((3, 12)); mv = np.zeros(12); mxi = np.zeros(4)
        fl = lib().oracle_moments(ctypes.byref(self.P), _p(np.ascontiguousarray(W, dtype=np.float64)),
                                  _p(mu), _p(mv), _p(mxi))
        return mu, mv, mxi, fl

    def micro_slope(self, W, b):
        a = np.zeros(self.nv)
        lib().oracle_micro_slope(ctypes.byref(self.P), _p(np.ascontiguousarray(W, dtype=np.float64)),
                                 _p(np.ascontiguousarray(b, dtype=np.float64)), _p(a))
        return a

    def smoothness(self, poly, deg):
        """Eq. 3.13 of a polynomial given by its 9 coefficients in xi."""
        p = np.zeros(9)
        p[:len(poly)] = poly
        return lib().oracle_smoothness(_p(p), deg)

    def recon(self, d, sig6):
        """ASE-DFF polynomial (9 coefficients in xi) of one cell and the branch taken."""
        poly = np.zeros(9)
        br = lib().oracle_recon(ctypes.byref(self.P), _p(self.T), _p(np.ascontiguousarray(d, dtype=np.float64)),
                                _p(np.ascontiguousarray(sig6, dtype=np.float64)), _p(poly))
        return poly, br
