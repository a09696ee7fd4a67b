"""Operation count of the FP64 oracle's S2O4 step (test infrastructure only).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: ``tests/`` and the
measurement leg of ``bench.py`` may use it, the product path never does.

The method's floating-point work per cell-stage, counted, not estimated: one
whole S2O4 step of the oracle runs with

* its C part (reconstruction, DFF, kinetic weighting, flux and interface
  state at every face Gauss point) compiled as ``flopcount.cpp``, where every
  ``double`` is a scalar type that tallies additions, multiplications,
  divisions and special functions;
* its numpy part (the two-stage combination of Eq. 2.19-2.25 and the Gauss
  sums of the update) on arrays that tally every elementwise operation.

The tally of a whole step on an n x n mesh is c2 n^2 + c1 n + c0 (interior
work, boundary halos, set-up such as the Step 3 weights); three mesh sizes
give c2, the operations per cell and step, halved for a cell-stage.  The
oracle is a plain transcription (elimination for every micro-slope, moments
by generic expansion), so this counts the method as the paper states it, not
the fewest operations that reach the same numbers.
"""
import ctypes

import numpy as np

from . import DFF_LAG_STEP, Oracle, OParams, _p, build_tally

_lib = None
_COUNTED_UFUNCS = {np.add, np.subtract, np.multiply, np.true_divide, np.negative, np.power,
                   np.square, np.absolute, np.sqrt}


def _clib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_tally())
        dp = ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(OParams)
        ip = ctypes.POINTER(ctypes.c_int)
        _lib.oracle_faces_1d.argtypes = [P, dp, dp, dp, dp, dp, ctypes.c_double, dp, dp, ip, ip]
        _lib.oracle_faces_2d.argtypes = [P, dp, dp, ctypes.c_int, dp, dp, dp, dp, dp, dp, dp,
                                         ctypes.c_double, dp, dp, ip]
        _lib.oracle_tally_get.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)]
        _lib.oracle_point_2d.argtypes = [P, dp, dp, ctypes.c_double, dp]
    return _lib


class _Counted(np.ndarray):
    """ndarray whose elementwise arithmetic and einsum contractions are tallied."""
    ops = 0

    def __array_ufunc__(self, ufunc, method, *inputs, **kw):
        args = [np.asarray(x) if isinstance(x, _Counted) else x for x in inputs]
        if "out" in kw:
            kw["out"] = tuple(np.asarray(x) if isinstance(x, _Counted) else x for x in kw["out"])
        res = getattr(ufunc, method)(*args, **kw)
        if ufunc in _COUNTED_UFUNCS:
            if method == "__call__":
                _Counted.ops += int(np.size(res))
            elif method == "reduce":
                _Counted.ops += int(np.size(args[0]))
        if isinstance(res, np.ndarray):
            return res.view(_Counted)
        return res

    def __array_function__(self, func, types, args, kwargs):
        plain = [np.asarray(a) if isinstance(a, _Counted) else a for a in args]
        res = func(*plain, **kwargs)
        if func is np.einsum:
            # one multiply and one add per element of the operand product
            ops = [np.asarray(a) for a in plain[1:]]
            _Counted.ops += 2 * int(max(np.size(o) for o in ops))
        elif func is np.mean:
            _Counted.ops += int(np.size(plain[0]))
        if isinstance(res, np.ndarray):
            return res.view(_Counted)
        return res


class _TallyOracle(Oracle):
    """The oracle with its C part taken from the counting build."""

    def faces(self, dt, state=None):
        L = _clib()
        W, Wx, Wy, Wxl, Wyl = state if state is not None else (self.W, self.Wx, self.Wy, self.Wxl, self.Wyl)
        c = lambda a: None if a is None else np.ascontiguousarray(np.asarray(a))
        W, Wx, Wy, Wxl, Wyl = c(W), c(Wx), c(Wy), c(Wxl), c(Wyl)
        nx, ny, m = self.nx, self.ny, self.m
        ox = np.zeros((5, 4, ny, nx + 1, m))
        sgx = np.zeros((ny, nx + 1, m))
        oy = np.zeros((5, 4, ny + 1, nx, m))
        sgy = np.zeros((ny + 1, nx, m))
        args = (_p(W), _p(Wx), _p(Wy), _p(Wxl), _p(Wyl), _p(c(self.sx)), _p(c(self.sy)), dt)
        for d, (o, sg) in enumerate(((ox, sgx), (oy, sgy))):
            nf = ctypes.c_int(0)
            self.flags |= L.oracle_faces_2d(ctypes.byref(self.P), _p(self.T), _p(self.gx), d, *args, _p(o), _p(sg),
                                            ctypes.byref(nf))
        return tuple(a.view(_Counted) for a in (ox, sgx, oy, sgy))


def _step_tally(order, n, sigma):
    from paper_2508_13705_gb300 import inputs
    o = _TallyOracle(2, order, n, n, extent=(0.0, 2.0, 0.0, 2.0), dff_lag=DFF_LAG_STEP)
    st = inputs.density_wave_2d(n, order)
    sx = sy = None
    if sigma is not None:
        sx, sy = np.full((n, n + 1), sigma), np.full((n + 1, n), sigma)
    o.set_state(*st, sigma_x=sx, sigma_y=sy)
    for name in ("W", "Wx", "Wy", "Wxl", "Wyl", "sx", "sy"):
        setattr(o, name, getattr(o, name).view(_Counted))
    L = _clib()
    L.oracle_tally_reset()
    _Counted.ops = 0
    o.step(0.3 * (2.0 / n))
    t = (ctypes.c_ulonglong * 10)()
    L.oracle_tally_get(t)
    c = np.array(list(t), dtype=np.float64)
    c[0] += _Counted.ops  # numpy arithmetic joins the add class (both tallies)
    c[7] += _Counted.ops
    return c, o


def operations_per_cell_stage(order, branch="linear"):
    """Operations per cell and stage of the 2-D S2O4 step at `order`.

    branch "linear": smooth data, every stencil takes the highest linear
    branch (the paper's smooth tests and the benchmark vortex); "ao": the DFF
    strength set to 10 on every face, so every reconstruction takes the
    HWENO-AO branch (Algorithm 1).  Returns a dict with the floating-point
    operations per cell-stage, "flops" (add + mul + div with non-trivial
    operands) and "flops_all" (every operation the oracle executes), and the
    special-function calls.
    """
    sig = None if branch == "linear" else 10.0
    sizes = (8, 12, 16)
    rows = []
    for n in sizes:
        c, o = _step_tally(order, n, sig)
        rows.append(c)
    A = np.array([[n * n, n, 1.0] for n in sizes])
    coef = np.linalg.solve(A, np.array(rows))[0] / 2.0  # per cell, per stage
    names = ("add", "mul", "div", "sqrt", "exp", "erfc", "pow", "add_nt", "mul_nt", "div_nt")
    out = {k: round(float(v), 1) for k, v in zip(names, coef)}
    out["flops_all"] = round(float(coef[0] + coef[1] + coef[2]), 1)
    out["flops"] = round(float(coef[7] + coef[8] + coef[9]), 1)
    out["special"] = round(float(coef[3:7].sum()), 1)
    out["order"] = order
    out["branch"] = branch
    return out


def operations_per_face_point(order, tau_mode=0):
    """Operations of the kinetic part alone (Step 4, Eq. 2.6-2.8 and the time
    integrals) at one 2-D face Gauss point with unequal smooth states: the
    share of the flux kernel.  Same fields as operations_per_cell_stage, per
    point."""
    o = Oracle(2, order, 8, 8, tau_mode=tau_mode)
    rng = np.random.default_rng(1)

    def side(r, u, v, p):
        D = np.zeros((6, 4))
        D[0] = [r, r * u, r * v, p / 0.4 + 0.5 * r * (u * u + v * v)]
        D[1:] = 0.1 * rng.normal(size=(5, 4))
        return D

    Dl, Dr = side(1.0, 0.3, -0.2, 1.0), side(0.98, 0.31, -0.19, 1.01)
    out = np.zeros((5, 4))
    L = _clib()
    L.oracle_tally_reset()
    L.oracle_point_2d(ctypes.byref(o.P), _p(Dl), _p(Dr), 0.01, _p(out))
    t = (ctypes.c_ulonglong * 10)()
    L.oracle_tally_get(t)
    c = np.array(list(t), dtype=np.float64)
    names = ("add", "mul", "div", "sqrt", "exp", "erfc", "pow", "add_nt", "mul_nt", "div_nt")
    res = {k: float(v) for k, v in zip(names, c)}
    res["flops_all"] = float(c[0] + c[1] + c[2])
    res["flops"] = float(c[7] + c[8] + c[9])
    res["special"] = float(c[3:7].sum())
    return res


if __name__ == "__main__":
    import json
    for order in (5, 7, 9):
        for br in ("linear", "ao"):
            print(json.dumps(operations_per_cell_stage(order, br)))
