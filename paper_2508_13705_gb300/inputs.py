"""Seeded synthetic inputs: initial cell averages, cell slopes and line slopes.

This module holds none of the scheme's arithmetic.  It only evaluates given
initial flow fields and integrates them over cells and faces by tensor
Gauss-Legendre quadrature, producing the state the scheme starts from:

* W      cell averages of (rho, rho U[, rho V], rho E)          [nvar][ny][nx]
* Wx, Wy cell averages of the x / y derivatives                 [nvar][ny][nx]
* Wx_line[l] = (W(x_{i+1/2}, y_{j_l}) - W(x_{i-1/2}, y_{j_l})) / dx
  (line-averaged x slope on the l-th Gauss line of the cell)    [m][nvar][ny][nx]
* Wy_line likewise in y on the x Gauss lines.

Both the CUDA path's tests and the oracle receive the same arrays from here.
Workloads (shapes follow the paper's test problems):

* ``density_wave_1d``   Sec. 4.1 advection, rho = 1 + 0.2 sin(pi x), u = p = 1
* ``riemann_1d``        Sec. 4.2 shock tubes (Sod, Lax, ...)
* ``shu_osher_1d``      Sec. 4.3 shock / entropy-wave interaction on [-5, 5]
* ``density_wave_2d``   Sec. 4.6 advection, rho = 1 + 0.2 sin(pi (x + y))
* ``vortex_2d``         isentropic vortex (strength 5) on periodic [0, 10]^2
* ``quadrants_2d``      four-quadrant Riemann problem, seeded random states
* ``batch_2d``          seeded uneven meshes: Fourier modes + planar shock
* ``double_mach``       Sec. 4.8 double Mach reflection, with its boundary sides
* ``oblique_shock``     its Mach 10 shock alone, translating between inflow sides
"""
import numpy as np


def _gl(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * x, 0.5 * w


def line_nodes(order):
    """Gauss lines per cell: 2, 3, 4 for orders 5, 7, 9; nodes on [-1/2, 1/2]."""
    m = {5: 2, 7: 3, 9: 4}[order]
    return _gl(m)[0]


def _cons(rho, u, v, p, gamma, dim):
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    if dim == 1:
        return np.stack([rho, rho * u, E])
    return np.stack([rho, rho * u, rho * v, E])


# ---------------------------------------------------------------------- 1-D

def cell_state_1d(prim, nx, x0, x1, gamma=1.4, nq=8):
    """prim(x) -> (rho, u, p) arrays.  Returns W, Wx ([3][1][nx])."""
    dx = (x1 - x0) / nx
    xc = x0 + (np.arange(nx) + 0.5) * dx
    q, w = _gl(nq)
    W = np.zeros((3, nx))
    for k in range(nq):
        r, u, p = prim(xc + q[k] * dx)
        W += w[k] * _cons(r, u, 0 * r, p, gamma, 1)
    r, u, p = prim(xc + 0.5 * dx)
    Wr = _cons(r, u, 0 * r, p, gamma, 1)
    r, u, p = prim(xc - 0.5 * dx)
    Wl = _cons(r, u, 0 * r, p, gamma, 1)
    Wx = (Wr - Wl) / dx
    return W.reshape(3, 1, nx), Wx.reshape(3, 1, nx)


def density_wave_1d(nx, x0=0.0, x1=2.0, gamma=1.4, amp=0.2):
    """Sec. 4.1: rho = 1 + amp sin(pi x), u = 1, p = 1 (exact cell averages)."""
    return cell_state_1d(lambda x: (1 + amp * np.sin(np.pi * x), 1 + 0 * x, 1 + 0 * x), nx, x0, x1, gamma)


def density_wave_1d_exact_avg(nx, t, x0=0.0, x1=2.0, amp=0.2):
    """Exact cell averages of rho at time t for the 1-D advection problem."""
    dx = (x1 - x0) / nx
    xl = x0 + np.arange(nx) * dx - t
    return 1.0 + amp * (np.cos(np.pi * xl) - np.cos(np.pi * (xl + dx))) / (np.pi * dx)


def riemann_1d(nx, left, right, x0=0.0, x1=1.0, xs=0.5, gamma=1.4):
    """Piecewise-constant (rho, u, p) with the jump on a cell face; zero slopes."""
    dx = (x1 - x0) / nx
    xc = x0 + (np.arange(nx) + 0.5) * dx
    lm = xc < xs
    prim = [np.where(lm, left[k], right[k]) for k in range(3)]
    W = _cons(prim[0], prim[1], 0 * prim[0], prim[2], gamma, 1)
    return W.reshape(3, 1, nx), np.zeros((3, 1, nx))


SOD = ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
LAX = ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571))


def shu_osher_1d(nx, gamma=1.4, x0=-5.0, x1=5.0, xs=-4.0):
    """Sec. 4.3 shifted to [-5, 5]: Mach-3 shock at x = -4 into rho = 1 + 0.2 sin 5x.

    Returns W, Wx and the fixed-profile ghost cells of the right end
    ([2 sides][3 layers][2 fields][3 vars]; the left side is unused).
    """
    left = (3.857143, 2.629369, 10.33333)

    def prim(x):
        lm = x < xs
        rho = np.where(lm, left[0], 1.0 + 0.2 * np.sin(5.0 * x))
        return rho, np.where(lm, left[1], 0.0), np.where(lm, left[2], 1.0)

    dx = (x1 - x0) / nx
    W, Wx = cell_state_1d(prim, nx, x0, x1, gamma)
    # the cells left of the jump are uniform: zero slopes there
    xc = x0 + (np.arange(nx) + 0.5) * dx
    Wx[:, 0, xc < xs] = 0.0
    ghost = np.zeros((2, 3, 2, 3))
    gW, gWx = cell_state_1d(prim, 3, x1, x1 + 3 * dx, gamma)
    ghost[1, :, 0, :] = gW[:, 0, :].T
    ghost[1, :, 1, :] = gWx[:, 0, :].T
    lW, _ = cell_state_1d(prim, 3, x0 - 3 * dx, x0, gamma)
    ghost[0, :, 0, :] = lW[:, 0, ::-1].T
    return W, Wx, ghost


# ---------------------------------------------------------------------- 2-D

def cell_state_2d(prim, nx, ny, extent, order, gamma=1.4, nq=6, rows_per_chunk=None):
    """prim(x, y) -> (rho, u, v, p).  Returns W, Wx, Wy, Wx_line, Wy_line (float64)."""
    x0, x1, y0, y1 = extent
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
    q, w = _gl(nq)
    gl = line_nodes(order)
    m = len(gl)
    W = np.zeros((4, ny, nx))
    Wx = np.zeros((4, ny, nx))
    Wy = np.zeros((4, ny, nx))
    Wxl = np.zeros((m, 4, ny, nx))
    Wyl = np.zeros((m, 4, ny, nx))
    xc = x0 + (np.arange(nx) + 0.5) * dx
    chunk = rows_per_chunk or max(1, min(ny, 2 ** 22 // max(1, nx * nq)))

    def cons(x, y):
        r, u, v, p = prim(x, y)
        return _cons(r, u, v, p, gamma, 2)

    for j0 in range(0, ny, chunk):
        j1 = min(ny, j0 + chunk)
        yc = y0 + (np.arange(j0, j1) + 0.5) * dy
        Y, X = np.meshgrid(yc, xc, indexing="ij")
        for a in range(nq):
            for b in range(nq):
                W[:, j0:j1] += w[a] * w[b] * cons(X + q[b] * dx, Y + q[a] * dy)
            # face averages for the cell-averaged slopes
            Wx[:, j0:j1] += w[a] * (cons(X + 0.5 * dx, Y + q[a] * dy) - cons(X - 0.5 * dx, Y + q[a] * dy)) / dx
            Wy[:, j0:j1] += w[a] * (cons(X + q[a] * dx, Y + 0.5 * dy) - cons(X + q[a] * dx, Y - 0.5 * dy)) / dy
        for l in range(m):
            Wxl[l, :, j0:j1] = (cons(X + 0.5 * dx, Y + gl[l] * dy) - cons(X - 0.5 * dx, Y + gl[l] * dy)) / dx
            Wyl[l, :, j0:j1] = (cons(X + gl[l] * dx, Y + 0.5 * dy) - cons(X + gl[l] * dx, Y - 0.5 * dy)) / dy
    return W, Wx, Wy, Wxl, Wyl


def density_wave_2d(n, order, gamma=1.4, amp=0.2):
    """Sec. 4.6: rho = 1 + amp sin(pi (x + y)), U = (1, 1), p = 1 on [0, 2]^2."""
    f = lambda x, y: (1 + amp * np.sin(np.pi * (x + y)), 1 + 0 * x, 1 + 0 * x, 1 + 0 * x)
    return cell_state_2d(f, n, n, (0.0, 2.0, 0.0, 2.0), order, gamma)


def density_wave_2d_exact_avg(n, t, amp=0.2):
    """Exact cell averages of rho(x, y, t) = 1 + amp sin(pi (x + y - 2t)) on [0,2]^2.

    With U = (1, 1) the profile moves along the diagonal, so the phase is
    x + y - 2t (Sec. 4.6 prints x + y - t; both agree at t = 2).
    """
    h = 2.0 / n
    xl = np.arange(n) * h
    A = xl[None, :] + xl[:, None] - 2.0 * t
    # average of sin(pi (x + y + c)) over a cell: product of sinc-type factors
    s = (np.sin(np.pi * (A + 2 * h)) - 2 * np.sin(np.pi * (A + h)) + np.sin(np.pi * A))
    return 1.0 - amp * s / (np.pi * h) ** 2


def vortex_prim(gamma=1.4, eps=5.0, xc=5.0, yc=5.0):
    def f(x, y):
        dxp, dyp = x - xc, y - yc
        r2 = dxp * dxp + dyp * dyp
        e = np.exp(0.5 * (1.0 - r2))
        u = 1.0 - eps / (2 * np.pi) * e * dyp
        v = 1.0 + eps / (2 * np.pi) * e * dxp
        T = 1.0 - (gamma - 1.0) * eps ** 2 / (8 * gamma * np.pi ** 2) * e * e
        rho = T ** (1.0 / (gamma - 1.0))
        return rho, u, v, rho * T
    return f


def vortex_2d(n, order, gamma=1.4, nq=6):
    """Isentropic vortex of strength 5 at (5, 5) on periodic [0, 10]^2, background (1,1,1,1)."""
    return cell_state_2d(vortex_prim(gamma), n, n, (0.0, 10.0, 0.0, 10.0), order, gamma, nq=nq)


def quadrant_states(seed=0, gamma=1.4):
    """Seeded quadrant states (rho, u, v, p) for quadrants (SW, SE, NE, NW).

    Drawn uniformly (rho in [0.1,1.5], u,v in [-1,1], p in [0.03,1.5]) and
    redrawn until every pair of adjacent quadrants differs in pressure by at
    least 10% of the larger one or in normal velocity by at least 0.1, so each
    interface carries a shock or a rarefaction.
    """
    rng = np.random.default_rng(seed)
    pairs = [(0, 1, 0), (3, 2, 0), (0, 3, 1), (1, 2, 1)]  # (a, b, axis of the normal)
    while True:
        s = np.stack([rng.uniform(0.1, 1.5, 4), rng.uniform(-1, 1, 4), rng.uniform(-1, 1, 4),
                      rng.uniform(0.03, 1.5, 4)], axis=1)
        ok = True
        for a, b, ax in pairs:
            dp = abs(s[a, 3] - s[b, 3]) / max(s[a, 3], s[b, 3])
            dun = abs(s[a, 1 + ax] - s[b, 1 + ax])
            ok &= dp >= 0.1 or dun >= 0.1
        if ok:
            return s


# Sec. 4.7: the four-quadrant states (rho, u, v, p) of Configurations 2 and 3
# for quadrants (SW, SE, NE, NW) and the split point.
CONFIG2 = (np.array([[1.0, -0.7259, -0.7259, 1.0], [0.5197, 0.0, -0.7259, 0.4], [1.0, 0.0, 0.0, 1.0],
                     [0.5197, -0.7259, 0.0, 0.4]]), (0.5, 0.5))
CONFIG3 = (np.array([[0.138, 1.206, 1.206, 0.029], [0.5323, 0.0, 1.206, 0.3], [1.5, 0.0, 0.0, 1.5],
                     [0.5323, 1.206, 0.0, 0.3]]), (0.7, 0.7))


def quadrants_2d(n, order, seed=0, gamma=1.4, split=(0.5, 0.5), states=None):
    """Four-quadrant Riemann problem on [0,1]^2 (split on cell faces); zero
    slopes.  ``states`` (SW, SE, NE, NW rows of rho, u, v, p) defaults to the
    seeded draw of quadrant_states(seed)."""
    s = quadrant_states(seed, gamma) if states is None else np.asarray(states, dtype=float)
    h = 1.0 / n
    xc = (np.arange(n) + 0.5) * h
    east = (xc >= split[0])[None, :]
    north = (xc >= split[1])[:, None]
    q = np.where(north, np.where(east, 2, 3), np.where(east, 1, 0))
    prim = s[q]  # [ny][nx][4]
    W = _cons(prim[..., 0], prim[..., 1], prim[..., 2], prim[..., 3], gamma, 2)
    m = len(line_nodes(order))
    z = np.zeros((4, n, n))
    return (np.ascontiguousarray(W), z.copy(), z.copy(), np.zeros((m, 4, n, n)), np.zeros((m, 4, n, n)))


def rankine_hugoniot(mach, rho1=1.0, p1=1.0, gamma=1.4):
    """Post-shock (rho, un, p) behind a shock of Mach ``mach`` moving into gas at rest."""
    g = gamma
    a1 = np.sqrt(g * p1 / rho1)
    M2 = mach * mach
    rho2 = rho1 * (g + 1) * M2 / ((g - 1) * M2 + 2)
    p2 = p1 * (2 * g * M2 - (g - 1)) / (g + 1)
    u2 = mach * a1 * (1 - rho1 / rho2)
    return rho2, u2, p2


def batch_specs(count=256, seed=0, lo=64, hi=512):
    """Seeded uneven batch: per instance nx, ny, modes, phases, shock Mach/position/axis."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(count):
        nx, ny = int(rng.integers(lo, hi + 1)), int(rng.integers(lo, hi + 1))
        a = rng.uniform(0, 1, 4)
        a = a / a.sum()
        kv = rng.integers(1, 5, size=(4, 2))
        ph = rng.uniform(0, 2 * np.pi, 4)
        mach = rng.uniform(1.5, 3.0)
        axis = int(rng.integers(0, 2))
        pos = rng.uniform(0.2, 0.8)
        specs.append(dict(nx=nx, ny=ny, a=a, k=kv, phase=ph, mach=mach, axis=axis, pos=pos))
    return specs


def batch_instance(spec, order, gamma=1.4, nq=4):
    """One batch member: smooth density modes on rho = 1, p = 1 plus a planar shock.

    The domain is [0,1] x [0, ny/nx] (square cells), periodic.  The shock front
    is snapped to a cell face; the post-shock side is uniform (zero slopes).
    """
    nx, ny = spec["nx"], spec["ny"]
    Ly = ny / nx
    h = 1.0 / nx
    ax = spec["axis"]
    ncell = nx if ax == 0 else ny
    xs = round(spec["pos"] * ncell) * h
    r2, u2, p2 = rankine_hugoniot(spec["mach"], gamma=gamma)

    def prim(x, y):
        rho = 1.0 + 0 * x
        for k in range(4):
            kx, ky = spec["k"][k]
            rho = rho + 0.2 * spec["a"][k] * np.sin(2 * np.pi * (kx * x + ky * y / Ly) + spec["phase"][k])
        c = x if ax == 0 else y
        post = c < xs
        rho = np.where(post, r2, rho)
        un = np.where(post, u2, 0.0)
        p = np.where(post, p2, 1.0)
        return (rho, un, 0 * x, p) if ax == 0 else (rho, 0 * x, un, p)

    W, Wx, Wy, Wxl, Wyl = cell_state_2d(prim, nx, ny, (0.0, 1.0, 0.0, Ly), order, gamma, nq=nq)
    # cells behind the front are uniform; the front sits on a face
    coord = (np.arange(ncell) + 0.5) * h
    post = coord < xs
    if ax == 0:
        sl = (slice(None), slice(None), post)
        for A in (Wx, Wy):
            A[sl] = 0.0
        Wxl[:, :, :, post] = 0.0
        Wyl[:, :, :, post] = 0.0
    else:
        Wx[:, post, :] = 0.0
        Wy[:, post, :] = 0.0
        Wxl[:, :, post, :] = 0.0
        Wyl[:, :, post, :] = 0.0
    return W, Wx, Wy, Wxl, Wyl


# Boundary codes of the C ABI (the oracle uses the same numbers)
_BC_TRANSMISSIVE, _BC_INFLOW, _BC_INFLOW_REFLECTIVE = 1, 5, 6
# Mach 10 shock of Sec. 4.8: speed 10 into gas at rest (sound speed 1), its
# front at 60 degrees to the x axis, so it crosses every horizontal line at
# 10 / sin 60 = 20 / sqrt 3
SHOCK_SPEED_X = 20.0 / np.sqrt(3.0)


def _mach10_states(gamma):
    s3 = np.sqrt(3.0)
    pre = np.asarray(_cons(1.4, 0.0, 0.0, 1.0, gamma, 2), dtype=np.float64)
    post = np.asarray(_cons(8.0, 4.125 * s3, -4.125, 116.5, gamma, 2), dtype=np.float64)
    return pre, post


def _oblique_shock(nx, ny, extent, xa, order, gamma):
    """Cell states (by the cell centre, zero slopes) of the Mach 10 shock whose
    front passes through (xa, 0) at 60 degrees: post-shock gas left of it."""
    pre, post = _mach10_states(gamma)
    x0, x1, y0, y1 = extent
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    xc = x0 + (np.arange(nx) + 0.5) * hx
    yc = y0 + (np.arange(ny) + 0.5) * hy
    ahead = yc[:, None] < np.sqrt(3.0) * (xc[None, :] - xa)
    W = np.where(ahead[None], pre.reshape(4, 1, 1), post.reshape(4, 1, 1))
    m = len(line_nodes(order))
    z = np.zeros((4, ny, nx))
    return (np.ascontiguousarray(W), z.copy(), z.copy(), np.zeros((m, 4, ny, nx)), np.zeros((m, 4, ny, nx)))


def double_mach(nx, ny, order, gamma=1.4):
    """Double Mach reflection (Sec. 4.8) on [0,4] x [0,1]: a Mach 10 shock
    through (1/6, 0) at 60 degrees to the x axis, gas at rest (1.4, 0, 0, 1)
    ahead of it and (8, 4.125 sqrt 3, -4.125, 116.5) behind; cell states by the
    cell centre, zero slopes.  Returns the state tuple and the boundary
    keywords: inflow of the post-shock state on the left, transmissive right,
    post-shock state below x = 1/6 and a slip wall beyond it at the bottom,
    and at the top the exact shock position 1/6 + (1 + 20 t) / sqrt 3 splitting
    post-shock from pre-shock ghost cells."""
    extent = (0.0, 4.0, 0.0, 1.0)
    state = _oblique_shock(nx, ny, extent, 1.0 / 6.0, order, gamma)
    pre, post = _mach10_states(gamma)
    bc_state = [[post, post], [post, post], [post, post], [post, pre]]
    bc_split = [[0.0, 0.0], [0.0, 0.0], [1.0 / 6.0, 0.0], [1.0 / 6.0 + 1.0 / np.sqrt(3.0), SHOCK_SPEED_X]]
    kw = dict(extent=extent, bc=(_BC_INFLOW, _BC_TRANSMISSIVE, _BC_INFLOW_REFLECTIVE, _BC_INFLOW),
              bc_state=np.asarray(bc_state, dtype=np.float64), bc_split=np.asarray(bc_split, dtype=np.float64))
    return state, kw


def oblique_shock(nx, ny, order, xa=0.3, height=0.5, speed=SHOCK_SPEED_X, gamma=1.4):
    """The Mach 10 shock of Sec. 4.8 alone, translating through [0,1] x
    [0,height] from (xa, 0): every side is an inflow side, left post-shock,
    right pre-shock, and below and above the shock's position on that side,
    xa + (y + 20 t) / sqrt 3, splits post- from pre-shock ghost cells (``speed``
    replaces 20 / sqrt 3 to move the split wrongly).  The exact solution is the
    translated shock."""
    extent = (0.0, 1.0, 0.0, height)
    state = _oblique_shock(nx, ny, extent, xa, order, gamma)
    pre, post = _mach10_states(gamma)
    bc_state = [[post, post], [pre, pre], [post, pre], [post, pre]]
    bc_split = [[0.0, 0.0], [0.0, 0.0], [xa, speed], [xa + height / np.sqrt(3.0), speed]]
    kw = dict(extent=extent, bc=(_BC_INFLOW,) * 4,
              bc_state=np.asarray(bc_state, dtype=np.float64), bc_split=np.asarray(bc_split, dtype=np.float64))
    return state, kw
