"""CPU-side checks of the C ABI library: it loads, exports every declared
symbol, validates parameters without a GPU, and its host table generator
reproduces the paper's printed stencil coefficients."""
import os
import re
from fractions import Fraction as Fr

import numpy as np
import pytest

from paper_2508_13705_gb300 import build, cgks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return cgks.lib()


def declared():
    txt = open(os.path.join(ROOT, "include", "cgks.h")).read()
    return sorted(set(re.findall(r"\b(cgks_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(L):
    names = declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(cgks.EXPORTS)


def test_invalid_parameters_rejected_without_gpu(L):
    import ctypes
    h = ctypes.c_void_p()
    for kw in (dict(order=6), dict(gamma=1.0), dict(cfl=0.0), dict(dim=3)):
        p = cgks.make_params(2, 9)
        for k, v in kw.items():
            setattr(p, k, v)
        assert L.cgks_init_mesh(ctypes.byref(h), ctypes.byref(p), 8, 8, 0.0, 1.0, 0.0, 1.0, None) == cgks.EINVAL
        assert not h.value
    p = cgks.make_params(2, 9)
    p.bc[0] = cgks.BC_FIXED  # fixed ghost cells are 1-D only
    assert L.cgks_init_mesh(ctypes.byref(h), ctypes.byref(p), 8, 8, 0.0, 1.0, 0.0, 1.0, None) == cgks.EINVAL
    p = cgks.make_params(2, 9)
    assert L.cgks_init_mesh(ctypes.byref(h), ctypes.byref(p), 0, 8, 0.0, 1.0, 0.0, 1.0, None) == cgks.EINVAL
    assert cgks.strerror(cgks.ENONPHYS).startswith("non-positive")


def test_size_limits_rejected_without_gpu(L):
    """Host-side limits, checked before any device call: a wall needs three
    cells to mirror its ghost layers onto; a mesh's work items are indexed in
    32 bits (2-D order 9 has 8 (n + 1) n face points at n x n); the point
    fallback is compiled into the tau > 0 flux only."""
    import ctypes
    h = ctypes.c_void_p()
    for bc, nx, ny in (((cgks.BC_REFLECTIVE, 0, 0, 0), 2, 8), ((0, 0, cgks.BC_NOSLIP, 0), 8, 2)):
        p = cgks.make_params(2, 9)
        for k in range(4):
            p.bc[k] = bc[k]
        assert L.cgks_init_mesh(ctypes.byref(h), ctypes.byref(p), nx, ny, 0.0, 1.0, 0.0, 1.0, None) == cgks.EINVAL
        assert not h.value
    n = 16385  # 8 * 16386 * 16385 >= 2^31 face points
    p = cgks.make_params(2, 9)
    assert 8 * (n + 1) * n >= 2 ** 31
    assert L.cgks_init_mesh(ctypes.byref(h), ctypes.byref(p), n, n, 0.0, 1.0, 0.0, 1.0, None) == cgks.EINVAL
    assert not h.value
    p = cgks.make_params(2, 9)
    p.pt_fallback = cgks.PT_FALLBACK_FIRST_ORDER  # with the default tau = 0
    assert L.cgks_init_mesh(ctypes.byref(h), ctypes.byref(p), 8, 8, 0.0, 1.0, 0.0, 1.0, None) == cgks.ENOTSUP
    assert not h.value


GOLD = os.path.join(ROOT, "tests", "golden", "stencils_eq3_8_3_10_3_18.txt")
ST = {"S0": 0, "S1": 1, "S2": 2, "r5": 3, "r7": 4, "r9": 5}


def test_host_tables_reproduce_printed_coefficients(L):
    """The library's own extended-precision generator against Eq. 3.8/3.10/3.18."""
    for line in open(GOLD):
        if not line.strip() or line.startswith("#"):
            continue
        f = line.split()
        for order in (5, 9):
            row = cgks.stencil_row(order, ST[f[0]], int(f[1]))
            for k, p in enumerate(f[2:]):
                want = -223 / 1260 if p == "omitted" else float(Fr(p))
                assert abs(row[k] - want) <= 1e-15 * max(1, abs(want)), (f[0], f[1], k)


def test_host_tables_gauss_rows_reproduce_polynomials(L):
    """Rows 6.. evaluate the r9 polynomial at the Gauss nodes: exact for data
    sampled from a degree-8 polynomial."""
    rng = np.random.default_rng(2)
    c = rng.normal(size=9)
    P = np.polynomial.Polynomial(c)
    I = P.integ()
    d = [I(k + 0.5) - I(k - 0.5) for k in range(-2, 3)] + [P(k + 0.5) - P(k - 0.5) for k in range(-2, 3)]
    for order, m in ((5, 2), (7, 3), (9, 4)):
        x = 0.5 * np.polynomial.legendre.leggauss(m)[0]
        for l in range(m):
            row = cgks.stencil_row(order, 5, 6 + l)
            assert abs(row @ d - P(x[l])) < 1e-12


def test_linear_stencils_use_only_their_taps(L):
    """The kernels skip, at compile time, the taps a linear stencil of Sec. 3.2
    does not use (the reconstructing cell's own gradient, and cells outside
    the stencil); the generated rows must vanish there.  The own-average tap
    (2) is nonzero in the rows but multiplies Qbar_i - Qbar_i = 0."""
    used = {3: {1, 3, 6, 8}, 4: {0, 1, 3, 4, 6, 8}, 5: {0, 1, 3, 4, 5, 6, 8, 9}}
    for order, m in ((5, 2), (7, 3), (9, 4)):
        for st, taps in used.items():
            for row in list(range(6)) + list(range(6, 6 + m)):
                r = cgks.stencil_row(order, st, row)
                for k in range(10):
                    if k not in taps and k != 2:
                        assert r[k] == 0.0, (order, st, row, k)
