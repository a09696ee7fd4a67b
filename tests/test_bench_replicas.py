"""The bench's multi-GPU path is replicas only: every rank runs the whole
workload on its own GPU, no data moves between ranks, and the whole-job rate
is the cell-stages of all ranks over the slowest rank's time.  This checks
that host logic (process-group set-up from the launcher's environment,
barrier, max and sum over ranks, the whole-job rate) with two gloo ranks on
the CPU."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    r, w, local, pg = bench.dist_setup(0)  # no GPUs: the gloo backend
    bench.barrier(pg)
    ms = 10.0 + r  # rank r "took" 10 + r ms for 1e6 (r + 1) cell-stages
    res = {"rank": r, "world": w, "local": local, "backend": pg.get_backend(),
           "max_ms": bench.max_over_ranks(pg, ms),
           "sum": bench.sum_over_ranks(pg, float(r + 1)),
           "rate": bench.whole_job_rate(pg, 1e6 * (r + 1), ms)}
    bench.barrier(pg)
    pg.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.json" % r), "w") as f:
        json.dump(res, f)


def test_replica_reductions_on_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    for r in range(world):
        res = json.load(open(tmp_path / ("rank%d.json" % r)))
        assert res["rank"] == r and res["world"] == world and res["local"] == r
        assert res["backend"] == "gloo"
        assert res["max_ms"] == 11.0
        assert res["sum"] == 3.0
        # 3e6 cell-stages in the slowest rank's 11 ms
        assert abs(res["rate"] - 3e6 / 11e-3 / 1e6) < 1e-9


def test_single_process_reductions_are_identities():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 4.5) == 4.5
    assert bench.sum_over_ranks(None, 2.0) == 2.0
    assert abs(bench.whole_job_rate(None, 2e6, 4.0) - 500.0) < 1e-12
