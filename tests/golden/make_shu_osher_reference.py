"""Write the reference solution of the Shu-Osher problem (Sec. 4.3; the
1-D shock-entropy configuration on [-5, 5] to t = 1.8) that the C2
measurements compare against: the FP64 CPU oracle, order 9, on 12800 cells
(CFL 0.5, HGKS collision time, transmissive left end, ghost cells fixed to
the initial profile at the right end), its cell averages of density averaged
conservatively onto 1600 cells (groups of 8).  Calls only the oracle and the
input generator; takes about an hour on eight cores.

    OMP_NUM_THREADS=8 python tests/golden/make_shu_osher_reference.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2508_13705_gb300 import inputs  # noqa: E402

N_REF, N_OUT, ORDER, T_END = 12800, 1600, 9, 1.8
OUT = os.path.join(HERE, "shu_osher_t1.8_rho_1600.txt")


def main():
    oracle.build()
    W, Wx, ghost = inputs.shu_osher_1d(N_REF)
    o = oracle.Oracle(1, ORDER, N_REF, extent=(-5.0, 5.0, 0.0, 1.0), tau_mode=oracle.TAU_HGKS,
                      bc=(oracle.BC_TRANSMISSIVE, oracle.BC_FIXED, 1, 1), cfl=0.5)
    o.set_state(W, Wx, ghost=ghost)
    t0 = time.time()
    steps = o.run(T_END)
    assert o.flags == 0 and abs(o.t - T_END) < 1e-12
    rho = o.W[0, 0].reshape(N_OUT, N_REF // N_OUT).mean(axis=1)
    with open(OUT, "w") as f:
        f.write("# Shu-Osher (Sec. 4.3) on [-5, 5], t = 1.8: density cell averages on %d cells,\n" % N_OUT)
        f.write("# the conservative average of the FP64 oracle at %d cells, order %d, CFL 0.5,\n" % (N_REF, ORDER))
        f.write("# HGKS collision time, transmissive left, fixed initial-profile ghosts right\n")
        f.write("# (%d steps, %.0f s); written by make_shu_osher_reference.py\n" % (steps, time.time() - t0))
        for v in rho:
            f.write("%.17e\n" % v)


if __name__ == "__main__":
    main()
