"""Checks on the stored Shu-Osher reference (Sec. 4.3; written by
tests/golden/make_shu_osher_reference.py from the FP64 oracle at 12800
cells) against what the problem itself fixes, independent of the scheme:

- the state left of the shock's starting point stays the uniform post-shock
  state (the left end is transmissive and the shock moves right);
- mass grows by exactly the inflow rho_L u_L t through the left end (the
  right end's ghosts hold the resting entropy wave, whose mass flux is zero
  up to the scheme's dissipation);
- the density ahead of the shock is still the resting entropy wave
  1 + 0.2 sin 5x (u = 0, p = 1 is a steady solution of the Euler equations);
- the shock, a Mach-3 shock into gas at rest with rho = 1, p = 1, travels at
  3 sqrt(gamma) and lies near x = -4 + 1.8 * 3 sqrt(1.4).
"""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
REF = os.path.join(HERE, "golden", "shu_osher_t1.8_rho_1600.txt")
LEFT = (3.857143, 2.629369, 10.33333)  # rho, u, p behind the shock
N, X0, X1, XS, T = 1600, -5.0, 5.0, -4.0, 1.8


def _ref():
    v = np.loadtxt(REF)
    assert v.shape == (N,)
    dx = (X1 - X0) / N
    xa = X0 + np.arange(N) * dx
    return v, xa, xa + dx, dx


def _wave_average(xa, xb):
    return 1.0 + 0.2 * (np.cos(5.0 * xa) - np.cos(5.0 * xb)) / (5.0 * (xb - xa))


def test_post_shock_state_kept_left_of_the_start():
    v, xa, xb, _ = _ref()
    assert np.abs(v[xb <= -4.5] - LEFT[0]).max() < 1e-10


def test_mass_grows_by_the_left_inflow():
    v, xa, xb, dx = _ref()
    m0 = LEFT[0] * (XS - X0) + (X1 - XS) + 0.2 * (np.cos(5.0 * XS) - np.cos(5.0 * X1)) / 5.0
    m1 = v.sum() * dx
    assert abs(m1 - (m0 + LEFT[0] * LEFT[1] * T)) < 1e-6 * m1


def test_resting_entropy_wave_ahead_of_the_shock():
    v, xa, xb, _ = _ref()
    ahead = xa >= 2.6
    assert np.abs(v[ahead] - _wave_average(xa[ahead], xb[ahead])).max() < 1e-4


def test_shock_position():
    v, xa, xb, _ = _ref()
    i = int(np.argmax(np.abs(np.diff(v))))
    x_shock = xb[i]
    assert abs(x_shock - (XS + T * 3.0 * np.sqrt(1.4))) < 0.05
    # the jump is a compression: dense behind, light ahead
    assert v[i] > 3.0 and v[i + 2] < 1.3
