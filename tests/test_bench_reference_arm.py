"""The bench's CPU legs, which need no GPU: the reference arm
(`--impl reference`, the FP64 oracle timed on the host cores) prints the
standard JSON line, and the worker the GPU arm's `cpu_baseline` spawns
reports its rate.  One oracle step of the 96^2 sample each."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BENCH = os.path.join(ROOT, "bench.py")


def _run(args, threads=4):
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    out = subprocess.check_output([sys.executable, BENCH] + args, env=env, text=True, timeout=600)
    return json.loads(out.strip().splitlines()[-1])


def test_reference_arm_line():
    line = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert line["impl"] == "reference"
    assert line["unit"] == "Mcell-stage/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 0
    assert line["dtype"] == "f64" and line["data"] == "synthetic"
    assert "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 4 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_cpu_worker_reports_rate():
    r = _run(["--cpu-worker", "1", "--order", "9"], threads=2)
    assert r["steps"] == 1 and r["seconds"] > 0
    assert abs(r["rate"] - 96 * 96 * 2 / r["seconds"] / 1e6) < 1e-9 * r["rate"] + 1e-12
