"""The operation counts bench.py divides by are the oracle's own tally
(oracle/tally.py, the oracle compiled with a counting scalar type): keep the
two in step whenever the oracle changes."""
import importlib.util
import os

import pytest

from oracle import tally

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_kinetic_point_counts_match_the_oracle_tally():
    b = _bench()
    assert tally.operations_per_face_point(9, 0)["flops"] == pytest.approx(b.ORACLE_FLOPS["kinetic_point_tau0"], abs=0.5)
    assert tally.operations_per_face_point(9, 1)["flops"] == pytest.approx(b.ORACLE_FLOPS["kinetic_point_tau"], abs=0.5)


@pytest.mark.parametrize("order", [5, 7, 9])
def test_cell_stage_counts_match_the_oracle_tally(order):
    b = _bench()
    got = tally.operations_per_cell_stage(order, "linear")["flops"]
    assert got == pytest.approx(b.ORACLE_FLOPS["cell_stage_linear"][order], abs=0.5)
