#!/usr/bin/env python
"""Throughput of the ASE-DFF compact gas-kinetic S2O4 step on GB300.

Workload (one "step" = one full two-stage S2O4 step of the whole mesh, CFL
time step computed on the device): 2-D Euler, gamma 1.4, periodic
[0,10]^2, isentropic vortex of strength 5 (background rho = u = v = p = 1),
ninth-order ASE-DFF(9,7,5,3), CFL 0.5, tau = 0, on 1024^2 cells.  Synthetic,
deterministic input generated by ``paper_2508_13705_gb300.inputs`` (cell
averages and slopes by Gauss quadrature of the analytic vortex).

Metric: Mcell-stage/s = cells x 2 stages x steps / device time, of the
FP32-bulk form at a fixed L1 error: the same run measures the L1 density
error of both forms against the exact solution after one period (t = 10) on
256^2, 512^2 and 1024^2, and the headline mesh is the finest of the vortex
meshes (1024^2, 2048^2) where the FP32-bulk error is within 10% of the plain
FP64 form's.  The FP64 form is timed on the same mesh (``fp64_plain``), and
the FP32 form also on 2048^2 (``fp32_2048``, reported with its accuracy
standing).  ``--impl reference`` times the FP64 CPU oracle instead.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
METRIC = "Mcell-stage/s 2D 9th-order, FP32 form vs FP64 plain at fixed L1 err; %roofline"

# The method's floating-point operations, counted by the FP64 oracle's
# operation-counting build (``python -m oracle.tally``; the test
# test_bench_constants checks these numbers against it): per face Gauss point
# of the kinetic part (Step 4, Eq. 2.6-2.8 and the time integrals; tau = 0,
# and with the collision terms for tau > 0), and per cell-stage of the whole
# 2-D step with every stencil on its highest linear branch.  Operations with
# a structural zero or +-1 operand are not counted.
ORACLE_FLOPS = {
    "kinetic_point_tau0": 9243.0, "kinetic_point_tau": 9573.0,
    "cell_stage_linear": {5: 40266.1, 7: 63046.3, 9: 88703.7},
}

# What the stage-1 flux kernel (order 9, tau = 0) executes per cell, counted
# by ncu on the 1024^2 vortex (FADD + FMUL + 2 FFMA, or the FP64
# counterparts; dram__bytes_read.sum + dram__bytes_write.sum), for the
# kernels as profiled in profiles/kernel_counters_vortex1024_o9.md: the pipe
# utilisation beside the algorithmic rate, and the DRAM traffic per launch.
FLUX1_EXECUTED = {"fp32": {"flops_per_cell": 20723.8, "dram_bytes_per_cell": 1417.5},
                  "fp64": {"flops_per_cell": 21389.3, "dram_bytes_per_cell": 2711.5}}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--order", type=int, default=9)
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-config3", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the orders, 4096^2 and Shu-Osher blocks")
    ap.add_argument("--cpu-worker", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--profile-case", choices=["fp32", "fp64"], default=None,
                    help="run one warm-up step and one step kernel by kernel on the --n vortex in the "
                         "given form, then exit (the small case the ncu captures use)")
    return ap.parse_args()


def profile_case(a):
    """Autotune, one warm-up S2O4 step, then one step launched kernel by kernel
    (no graph) inside the NVTX range `profiled`, on the n x n order-`order`
    vortex: the bench's launch shapes in a short launch sequence for ncu."""
    import torch

    from paper_2508_13705_gb300 import build, cgks
    build.build()
    st = vortex_inputs(a.n, a.order)
    prec = cgks.FP32_BULK if a.profile_case == "fp32" else cgks.FP64
    s = cgks.Solver(2, a.order, a.n, a.n, extent=(0.0, 10.0, 0.0, 10.0), precision=prec)
    s.set_state(*st)
    tuned = s.autotune()
    s.advance(1, 0.0)
    s.sync()
    dt = s.compute_dt()
    torch.cuda.nvtx.range_push("profiled")
    ms = s.profile_step(dt)
    s.sync()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile_case": a.profile_case, "n": a.n, "order": a.order,
                      "autotuned_threads": tuned, "kernels_ms": ms}))
    s.sync()
    s.close()
    torch.cuda.synchronize()


def dist_setup(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if n > 0 else "gloo")
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def _reduce(pg, x, op):
    import torch
    dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(pg, x):
    """The largest x over the ranks (this rank's x without a process group)."""
    return x if pg is None else _reduce(pg, x, pg.ReduceOp.MAX)


def sum_over_ranks(pg, x):
    return x if pg is None else _reduce(pg, x, pg.ReduceOp.SUM)


def whole_job_rate(pg, cell_stages, ms):
    """Mcell-stage/s of the whole job: the cell-stages every rank processed
    over the slowest rank's time (each rank passes its own count and ms)."""
    return sum_over_ranks(pg, float(cell_stages)) / (max_over_ranks(pg, ms) / 1e3) / 1e6


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def vortex_inputs(n, order):
    from paper_2508_13705_gb300 import inputs
    return inputs.vortex_2d(n, order)


def peaks():
    try:
        return json.load(open(HBM_PEAKS))
    except (OSError, ValueError):
        return {}


def nproc():
    try:
        return int(subprocess.check_output(["nproc"], text=True).strip())
    except (OSError, ValueError, subprocess.CalledProcessError):
        return os.cpu_count() or 1


KERNEL_NAMES = {0: "recon_x", 1: "recon_y", 2: "flux", 3: "update", 4: "dt"}


def kernel_ms(prof):
    return {(("s%d_" % (k // 10)) if k >= 10 else "") + KERNEL_NAMES[k % 10]: round(v, 4) for k, v in prof}


def timed_form(torch, cgks, st, n, order, precision, steps, warmup, stream, pg, tau_mode=0):
    """Autotuned solver, W warm-up steps, then K CFL steps timed by CUDA events
    on the solver's stream (barrier + synchronize on both sides)."""
    s = cgks.Solver(2, order, n, n, extent=(0.0, 10.0, 0.0, 10.0), precision=precision, tau_mode=tau_mode,
                    stream=stream.cuda_stream)
    s.set_state(*st)
    tuned = s.autotune()
    s.advance(warmup, 0.0)
    s.sync()
    barrier(pg)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed_" + ("fp32" if precision == cgks.FP32_BULK else "fp64"))
    e0.record(stream)
    s.advance(steps, 0.0)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()  # lets a profiler select the timed steps
    barrier(pg)
    ms = max_over_ranks(pg, e0.elapsed_time(e1))
    _, rc, _ = s.sync(raise_on_error=False)
    prof = kernel_ms(s.profile_step(s.compute_dt()))
    return s, ms, rc, tuned, prof


def main():
    a = parse()
    if a.cpu_worker:
        return cpu_worker(a)
    if a.impl == "reference":
        return reference_arm(a)
    if a.profile_case:
        return profile_case(a)
    import torch

    from paper_2508_13705_gb300 import build, cgks
    rank, world, local, pg = dist_setup(a.gpus)
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    barrier(pg)
    n, order = a.n, a.order
    t_in = time.perf_counter()
    st = vortex_inputs(n, order)
    t_in = time.perf_counter() - t_in
    stream = torch.cuda.Stream()
    cells = n * n
    extras = rank == 0 and world == 1  # the untimed measurements run at N = 1 only

    # ---------------- FP32-bulk form (headline), clocks sampled during the timed steps
    clk = ClockSampler(local)
    clk.start()
    s32, ms32, rc32, tuned32, prof32 = timed_form(torch, cgks, st, n, order, cgks.FP32_BULK, a.steps, a.warmup,
                                                 stream, pg)
    clocks = clk.stop()
    kps = s32.kernels_per_step()

    # ---------------- FP64 plain form, same mesh
    k64 = max(4, a.steps // 5)
    s64, ms64, rc64, tuned64, prof64 = timed_form(torch, cgks, st, n, order, cgks.FP64, k64, a.warmup, stream, pg)
    s64.close()

    # ---------------- end to end through the public API: the whole state from
    # pinned host arrays, one step, the state read back into them
    k_e2e = max(1, min(a.steps, 5))
    names = ("W", "Wx", "Wy", "Wx_line", "Wy_line", "sigma_x", "sigma_y")
    g = s32.get_state()
    pinned = {k: torch.from_numpy(g[k]).pin_memory() for k in names}
    host = {k: pinned[k].numpy() for k in names}
    bytes_state = sum(v.nbytes for v in host.values())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        s32.set_state(*[host[k] for k in names])
        s32.step(0.0)
        s32.get_state(out=host)  # straight into the pinned host buffers
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(pg, time.perf_counter() - t0)
    s32.close()

    value = whole_job_rate(pg, cells * 2 * a.steps, ms32)
    v64 = whole_job_rate(pg, cells * 2 * k64, ms64)
    e2e_v = whole_job_rate(pg, cells * 2 * k_e2e, e2e_s * 1e3)

    # ---------------- measured arithmetic peaks (FMA chains on every SM)
    p32, _ = cgks.fma_peak(cgks.FP32_BULK)
    p64, _ = cgks.fma_peak(cgks.FP64)
    hbm = peaks().get("hbm_gbs")

    line = {
        "metric": METRIC,
        "value": round(value, 3), "unit": "Mcell-stage/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(ms32 / a.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "isentropic vortex 2-D, periodic [0,10]^2, %dx%d cells, order %d, CFL 0.5, tau 0"
                               % (n, n, order),
                   "precision": "FP32 bulk over FP64 bases (cell averages, their accumulation, DFF and positivity "
                                "tests in FP64)",
                   "global_batch": world, "mesh": [n, n],
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (state %.2f GB per replica)" % (bytes_state / 1e9)},
        "roofline": roofline(prof32, "fp32", order, n, p32, p64, hbm),
        "clocks": clocks,
        "e2e": {"value": round(e2e_v, 3), "unit": "Mcell-stage/s", "h2d_bytes_per_step": bytes_state,
                "d2h_bytes_per_step": bytes_state, "steps": k_e2e},
        "gpu_launches": kps * a.steps,
        "status": rc32,
        "input_gen_s": round(t_in, 2),
        "peaks_measured": {"fp32_fma_tflops": round(p32, 2), "fp64_fma_tflops": round(p64, 3),
                           "hbm_gbs": hbm, "basis": "cgks_fma_peak (FMA chains on every SM, CUDA events, "
                                                    "clocks as found); HBM from MEASURED_PEAKS.json"},
        "fp64_plain": {"value": round(v64, 3), "unit": "Mcell-stage/s", "steps": k64,
                       "ms_per_step": round(ms64 / k64, 4), "status": rc64, "autotuned_threads": tuned64,
                       "roofline": roofline(prof64, "fp64", order, n, p32, p64, hbm)},
        "autotuned_threads_fp32": tuned32,
    }
    acc = None
    if extras and not a.no_accuracy:
        acc = accuracy(torch, cgks, order, stream, n)
        line["accuracy"] = acc
        line["fp32_2048"] = larger_mesh(torch, cgks, order, stream, pg, a)
    if extras and not a.no_batch:
        line["batch"] = batch_bench(torch, cgks, stream, p32)
    if extras and not a.no_config3:
        line["config3"] = config3_bench(torch, cgks, stream)
    if extras and not a.no_configs:
        line["orders"] = orders_bench(torch, cgks, stream, a)
        line["quadrants_4096"] = quadrants_bench(torch, cgks, stream)
        line["shu_osher"] = shu_osher_bench(cgks)
    if extras and not a.no_cpu:
        line["cpu_baseline"] = cpu_baseline(order)
    # the figures a truncated log tail must still show, last
    row = None if acc is None else next((r for r in acc["rows"] if r["mesh"][0] == n), None)
    line["summary"] = {
        "fp32_bulk": round(value, 3), "fp64_plain": round(v64, 3), "unit": "Mcell-stage/s", "mesh": n,
        "fp64_ms_per_step": round(ms64 / k64, 3), "fp64_status": rc64,
        "l1_fp32_over_fp64_t10": None if row is None else round(row["fp32_over_fp64"], 5),
        "fixed_l1_holds": None if row is None else row["within_10pct"],
        "roofline_frac": line["roofline"]["frac"], "fp64_roofline_frac": line["fp64_plain"]["roofline"]["frac"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def roofline(kms, precision, order, n, p32, p64, hbm):
    """The dominant kernel of the step: the stage-1 flux kernel (Steps 3-4 and
    the time-integrated flux at every face Gauss point).  Its algorithmic work
    is the oracle's count of the kinetic part per face Gauss point times the
    launch's 2 m n (n + 1) points; the peak is the measured FMA throughput of
    the kernel's precision.  The kernels reach the oracle's results with fewer
    operations (one Gram matrix per Maxwellian, closed-form micro-slopes), so
    this algorithmic rate can exceed what the pipe executes."""
    m = (order - 1) // 2
    pts = 2 * m * n * (n + 1)
    ms = kms["s1_flux"]
    total = sum(v for k, v in kms.items())
    alg = ORACLE_FLOPS["kinetic_point_tau0"] * pts
    peak = p32 if precision == "fp32" else p64
    ach = alg / (ms / 1e3) / 1e12
    ex = FLUX1_EXECUTED[precision] if order == 9 else None
    out = {"bound": "alu", "kernel": "k_flux, stage 1", "achieved": round(ach, 3), "peak": round(peak, 2),
           "unit": "TFLOP/s", "frac": round(ach / peak, 4),
           "traffic": None if ex is None else round(ex["dram_bytes_per_cell"] * n * n),
           "executed": None if ex is None else {
               "tflops": round(ex["flops_per_cell"] * n * n / (ms / 1e3) / 1e12, 3),
               "frac": round(ex["flops_per_cell"] * n * n / (ms / 1e3) / 1e12 / peak, 4),
               "basis": "ncu executed FP operations per cell of this kernel on the 1024^2 vortex "
                        "(profiles/kernel_counters_vortex1024_o9.md) x n^2 / launch time"},
           "algorithmic_flops_per_launch": alg,
           "basis": "oracle operation tally of the kinetic part, %.0f per face Gauss point x %d points; "
                    "peak: measured %s FMA throughput" % (ORACLE_FLOPS["kinetic_point_tau0"], pts, precision),
           "share_of_step": round(ms / total, 4), "kernels_ms": kms,
           "step_algorithmic_tflops": round(ORACLE_FLOPS["cell_stage_linear"][order] * n * n * 2 / (total / 1e3) / 1e12, 3)}
    return out


def accuracy(torch, cgks, order, stream, n_work, meshes=(256, 512, 1024), t_end=10.0):
    """L1 density error of both forms against the exact solution at t = 10 (one
    period, exact solution = the initial cell averages) on several meshes; the
    FP32-bulk form holds the fixed-L1 condition where its error is within 10%
    of the FP64 form's."""
    rows = [accuracy_one(torch, cgks, order, stream, n, t_end) for n in meshes]
    ok = [r["mesh"][0] for r in rows if r["within_10pct"]]
    return {"t": t_end, "rows": rows, "finest_mesh_within_10pct": max(ok) if ok else None}


def accuracy_one(torch, cgks, order, stream, n, t_end):
    st = vortex_inputs(n, order)
    out = {"mesh": [n, n], "t": t_end}
    for name, prec in (("fp64", cgks.FP64), ("fp32", cgks.FP32_BULK)):
        s = cgks.Solver(2, order, n, n, extent=(0.0, 10.0, 0.0, 10.0), precision=prec, stream=stream.cuda_stream)
        s.set_state(*st)
        t0 = time.perf_counter()
        t, steps, rc = s.run_to(t_end, max_steps=40000)
        W = s.get_state()["W"]
        out["l1_" + name] = float(np.abs(W[0] - st[0][0]).mean())
        out["status_" + name] = rc
        out["wall_s_" + name] = round(time.perf_counter() - t0, 1)
        out["steps"] = steps
        s.close()
    out["fp32_over_fp64"] = out["l1_fp32"] / out["l1_fp64"]
    out["within_10pct"] = bool(out["fp32_over_fp64"] <= 1.10)
    return out


def larger_mesh(torch, cgks, order, stream, pg, a):
    """The FP32-bulk form on the larger vortex mesh (2048^2): throughput, with
    the L1 errors of both forms after one period from a separate full run (the
    FP64 run there takes about 53 minutes, so the bench does not repeat it)."""
    n = 2048
    st = vortex_inputs(n, order)
    s, ms, rc, tuned, prof = timed_form(torch, cgks, st, n, order, cgks.FP32_BULK, a.steps, a.warmup, stream, pg)
    s.close()
    return {"mesh": [n, n], "value": round(n * n * 2 * a.steps / (ms / 1e3) / 1e6, 3), "unit": "Mcell-stage/s",
            "ms_per_step": round(ms / a.steps, 4), "status": rc, "kernels_ms": prof,
            "note": "not at fixed L1 error: after one period (t = 10, 13690 steps) FP32 bulk 1.111e-9 vs "
                    "FP64 9.329e-10 (ratio 1.19), measured in a separate full run of each form"}


def batch_bench(torch, cgks, stream, p32, count=256, order=7, steps=10):
    """Config C5: 256 seeded uneven periodic meshes (sides 64-512, smooth modes
    plus a planar shock), order 7, HGKS tau.  FP32-bulk batch (one persistent
    launch per kernel, one graph per step, device CFL per instance) timed over
    `steps` steps; the same instances stepped one at a time in FP64 over the
    same number of steps; and the relative L1 difference of the two after
    `steps` steps of fixed per-instance dt (the CFL step of the initial state)."""
    from paper_2508_13705_gb300 import inputs
    sp = inputs.batch_specs(count, seed=0)
    t0 = time.perf_counter()
    states = [inputs.batch_instance(s, order, nq=2) for s in sp]
    t_in = time.perf_counter() - t0
    nx = [s["nx"] for s in sp]
    ny = [s["ny"] for s in sp]
    ext = [(0.0, 1.0, 0.0, s["ny"] / s["nx"]) for s in sp]
    cells = sum(x * y for x, y in zip(nx, ny))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def make_batch():
        b = cgks.Batch(order, nx, ny, ext, precision=cgks.FP32_BULK, tau_mode=cgks.TAU_HGKS,
                       stream=stream.cuda_stream)
        for k, st in enumerate(states):
            b.set_state(k, *st)
        return b

    b = make_batch()
    tuned = b.autotune()
    for _ in range(2):
        b.step(None)
    b.sync()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        b.step(None)
    e1.record(stream)
    torch.cuda.synchronize()
    ms32 = e0.elapsed_time(e1)
    rc = 0
    try:
        b.sync()
    except cgks.CgksError as e:
        rc = e.code
    b.close()
    # fixed per-instance dt for the FP32-vs-FP64 comparison
    dts = []
    ms64 = 0.0
    fp64_final = []
    for k, st in enumerate(states):
        s = cgks.Solver(2, order, nx[k], ny[k], extent=ext[k], precision=cgks.FP64, tau_mode=cgks.TAU_HGKS,
                        stream=stream.cuda_stream)
        s.set_state(*st)
        dt = s.compute_dt()
        dts.append(dt)
        torch.cuda.synchronize()
        e0.record(stream)
        s.advance(steps, dt)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 += e0.elapsed_time(e1)
        fp64_final.append(s.get_state()["W"])
        s.close()
    b = make_batch()
    for _ in range(steps):
        b.step(np.array(dts))
    b.sync()
    num = den = 0.0
    worst = 0.0
    for k in range(count):
        W32 = b.get_state(k)["W"]
        d = np.abs(W32 - fp64_final[k]).sum()
        num += d
        den += np.abs(fp64_final[k]).sum()
        worst = max(worst, d / np.abs(fp64_final[k]).sum())
    b.close()
    value = cells * 2 * steps / (ms32 / 1e3) / 1e6
    alg = ORACLE_FLOPS["cell_stage_linear"][order] * cells * 2 * steps / (ms32 / 1e3) / 1e12
    return {"workload": "%d periodic instances, sides 64-512 (seed 0), Fourier modes + Mach 1.5-3 planar shock, "
                        "order %d, HGKS tau, CFL 0.5" % (count, order),
            "cells": cells,
            "fp32_batched": {"value": round(value, 3), "unit": "Mcell-stage/s", "steps": steps, "status": rc,
                             "autotuned_threads": tuned,
                             "roofline": {"bound": "alu", "achieved": round(alg, 3), "peak": round(p32, 2),
                                          "unit": "TFLOP/s", "frac": round(alg / p32, 4),
                                          "basis": "oracle operation tally per cell-stage at order %d (linear "
                                                   "branches) x cell-stages / step time; measured FP32 FMA peak"
                                                   % order}},
            "fp64_one_at_a_time": {"value": round(cells * 2 * steps / (ms64 / 1e3) / 1e6, 3),
                                   "unit": "Mcell-stage/s", "steps": steps},
            "fp32_batched_vs_fp64": {"rel_l1_W_all": num / den, "rel_l1_W_worst_instance": worst, "steps": steps,
                                     "dt": "per instance, the CFL step of its initial state"},
            "input_gen_s": round(t_in, 1)}


# The paper's CPU time (s) of the reconstruction alone over 20 steps of
# Configuration 3, one Xeon Gold 6133 core (the CPU-time table of Sec. 4),
# for orders 5, 7, 9 by mesh side.  Context only: other hardware, and a
# part of the step.
PAPER_RECON_CPU_S = {100: (0.913, 1.382, 1.942), 200: (5.244, 6.048, 7.685),
                     400: (15.764, 28.722, 30.228), 800: (63.766, 126.264, 119.484)}


def config3_bench(torch, cgks, stream, full_order=9):
    """Sec. 4.7 Configuration 3, the paper's timing workload: (1) 20 whole S2O4
    steps (CFL step on the device, HGKS tau, transmissive) at the four meshes
    of the paper's CPU-time table, FP64 and FP32 bulk, beside the paper's
    reconstruction-only CPU times; (2) the full run at 500^2 to t = 0.6 in the
    FP32-bulk form."""
    from paper_2508_13705_gb300 import inputs
    states, split = inputs.CONFIG3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def solver(n, order, prec):
        s = cgks.Solver(2, order, n, n, extent=(0.0, 1.0, 0.0, 1.0), precision=prec, tau_mode=cgks.TAU_HGKS,
                        bc=(1, 1, 1, 1), stream=stream.cuda_stream)
        s.set_state(*inputs.quadrants_2d(n, order, states=states, split=split))
        s.autotune()
        return s

    table = []
    for n, paper in PAPER_RECON_CPU_S.items():
        row = {"mesh": n, "paper_recon_cpu_s_orders_5_7_9": list(paper)}
        for prec, key in ((cgks.FP64, "fp64"), (cgks.FP32_BULK, "fp32")):
            ms = []
            for order in (5, 7, 9):
                s = solver(n, order, prec)
                torch.cuda.synchronize()
                e0.record(stream)
                s.advance(20, 0.0)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(round(e0.elapsed_time(e1), 3))
                _, rc, _ = s.sync(raise_on_error=False)
                s.close()
                if rc:
                    ms[-1] = None
            row[key + "_20_steps_ms_orders_5_7_9"] = ms
        table.append(row)
    s = solver(500, full_order, cgks.FP32_BULK)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t, steps, rc = s.run_to(0.6, max_steps=20000)
    wall = time.perf_counter() - t0
    s.close()
    full = {"steps": steps, "wall_s": round(wall, 3), "status": rc,
            "Mcell_stage_per_s": round(500 * 500 * 2 * steps / wall / 1e6, 3)}
    return {"workload": "2-D Riemann Configuration 3 (Sec. 4.7), transmissive, HGKS tau, CFL 0.5",
            "twenty_steps": table,
            "full_run_500_t0.6_order%d_fp32" % full_order: full,
            "note": "paper times: reconstruction only, one CPU core; GPU times: whole steps incl. CFL"}


def orders_bench(torch, cgks, stream, a, n=2048):
    """The vortex workload at 2048^2 at orders 5, 7 and 9, both forms (C3):
    device time per step over a few CFL steps after the autotuner."""
    from paper_2508_13705_gb300 import inputs
    out = {"mesh": [n, n]}
    for order in (5, 7, 9):
        st = inputs.cell_state_2d(inputs.vortex_prim(), n, n, (0.0, 10.0, 0.0, 10.0), order, nq=4)
        row = {}
        for name, prec, k in (("fp32", cgks.FP32_BULK, 10), ("fp64", cgks.FP64, 2)):
            s, ms, rc, tuned, prof = timed_form(torch, cgks, st, n, order, prec, k, 2, stream, None)
            s.close()
            row[name] = {"value": round(n * n * 2 * k / (ms / 1e3) / 1e6, 3), "ms_per_step": round(ms / k, 4),
                         "steps": k, "status": rc}
        out["order%d" % order] = row
    out["unit"] = "Mcell-stage/s"
    return out


def quadrants_bench(torch, cgks, stream, n=4096, order=9, steps=5):
    """C4: the seeded four-quadrant Riemann problem on [0,1]^2 at 4096^2, order
    9 with the DFF active, HGKS tau, transmissive, FP32 bulk: device time per
    CFL step and the branch counts of Algorithm 1 in the last step."""
    from paper_2508_13705_gb300 import inputs
    st = inputs.quadrants_2d(n, order, seed=0)
    s = cgks.Solver(2, order, n, n, extent=(0.0, 1.0, 0.0, 1.0), precision=cgks.FP32_BULK,
                    tau_mode=cgks.TAU_HGKS, bc=(1, 1, 1, 1), stream=stream.cuda_stream)
    s.set_state(*st)
    s.autotune()
    s.advance(2, 0.0)
    s.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.advance(steps, 0.0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    _, rc, _ = s.sync(raise_on_error=False)
    stats = s.stats()
    s.close()
    return {"workload": "four quadrants (seed 0), [0,1]^2, %dx%d, order %d, HGKS tau, transmissive, FP32 bulk"
                        % (n, n, order),
            "value": round(n * n * 2 * steps / (ms / 1e3) / 1e6, 3), "unit": "Mcell-stage/s",
            "ms_per_step": round(ms / steps, 3), "steps": steps, "status": rc,
            "branches_last_step": stats["branch"], "t": stats["t"]}


SHU_OSHER_REF = os.path.join(ROOT, "tests", "golden", "shu_osher_t1.8_rho_1600.txt")


def shu_osher_bench(cgks):
    """C2: the Shu-Osher problem (Sec. 4.3) to t = 1.8 on 400 and 1600 cells,
    orders 7 and 9, both forms: L1 density error against the 12800-cell oracle
    reference (tests/golden, averaged onto 1600 cells; onto 400 by groups of 4)."""
    from paper_2508_13705_gb300 import inputs
    if not os.path.exists(SHU_OSHER_REF):
        return {"unavailable": "reference file missing"}
    ref1600 = np.loadtxt(SHU_OSHER_REF)
    rows = []
    for N in (400, 1600):
        ref = ref1600.reshape(N, -1).mean(axis=1)
        for order in (7, 9):
            row = {"N": N, "order": order}
            for name, prec in (("fp64", cgks.FP64), ("fp32", cgks.FP32_BULK)):
                W, Wx, ghost = inputs.shu_osher_1d(N)
                s = cgks.Solver(1, order, N, extent=(-5.0, 5.0, 0.0, 1.0), precision=prec, tau_mode=cgks.TAU_HGKS,
                                bc=(cgks.BC_TRANSMISSIVE, cgks.BC_FIXED, 1, 1))
                s.set_ghost(ghost)
                s.set_state(W, Wx)
                t0 = time.perf_counter()
                t, steps, rc = s.run_to(1.8, max_steps=100000)
                wall = time.perf_counter() - t0
                rho = s.get_state()["W"][0, 0]
                s.close()
                row["l1_" + name] = float(np.abs(rho - ref).mean())
                row["status_" + name] = rc
                row["steps"] = steps
                row["wall_s_" + name] = round(wall, 2)
            row["fp32_over_fp64"] = row["l1_fp32"] / row["l1_fp64"]
            rows.append(row)
    return {"workload": "Shu-Osher, [-5,5], t = 1.8, HGKS tau, CFL 0.5; reference: oracle at 12800 cells",
            "rows": rows}


# ---------------------------------------------------------------- the oracle on the host cores

CPU_SAMPLE_N = 96


def cpu_worker(a):
    """Child process: time the FP64 oracle (as it stands) on the vortex problem
    at CPU_SAMPLE_N^2 over a given number of steps, with the OpenMP thread
    count the parent set."""
    import oracle
    oracle.build()
    steps = int(a.cpu_worker)
    n = CPU_SAMPLE_N
    st = vortex_inputs(n, a.order)
    o = oracle.Oracle(2, a.order, n, n, extent=(0.0, 10.0, 0.0, 10.0))
    o.set_state(*st)
    o.step()  # loads the library, warms the caches
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step()
    el = time.perf_counter() - t0
    print(json.dumps({"rate": n * n * 2 * steps / el / 1e6, "seconds": el, "steps": steps}), flush=True)


def _cpu_run(order, threads, steps):
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    out = subprocess.check_output([sys.executable, os.path.abspath(__file__), "--cpu-worker", str(steps),
                                   "--order", str(order)], env=env, text=True)
    return json.loads(out.strip().splitlines()[-1])


def cpu_baseline(order):
    """The FP64 oracle on the host: single-threaded and on all cores (nproc),
    each on a bounded sample of the same problem (the vortex at 96^2)."""
    cores = nproc()
    one = _cpu_run(order, 1, 2)
    allc = _cpu_run(order, cores, 10)
    sample = ("the %dx%d vortex problem (same physics and order as the GPU workload), one S2O4 step per step: "
              "%d step(s) single-threaded (%.1f s), %d steps on %d threads (%.1f s)"
              % (CPU_SAMPLE_N, CPU_SAMPLE_N, one["steps"], one["seconds"], allc["steps"], cores, allc["seconds"]))
    return {"value": round(allc["rate"], 5), "unit": "Mcell-stage/s", "cores": cores, "kind": "oracle",
            "sample": sample, "single_thread": {"value": round(one["rate"], 5), "cores": 1}}


def reference_arm(a):
    """The FP64 CPU oracle, timed on the host cores, on bounded samples."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    n_sample = CPU_SAMPLE_N
    order = a.order
    st = vortex_inputs(n_sample, order)
    o = oracle.Oracle(2, order, n_sample, n_sample, extent=(0.0, 10.0, 0.0, 10.0))
    o.set_state(*st)
    for _ in range(a.warmup):
        o.step()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        o.step()
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", nproc()))
    v = n_sample * n_sample * 2 * a.steps / el / 1e6
    sample = "the %dx%d vortex problem (same physics and order as the %d^2 workload), one S2O4 step per step" % (
        n_sample, n_sample, a.n)
    line = {"impl": "reference", "metric": METRIC,
            "value": round(v, 5), "unit": "Mcell-stage/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": round(el / a.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "isentropic vortex 2-D, periodic [0,10]^2, %dx%d cells, order %d, CFL 0.5, tau 0"
                                   % (a.n, a.n, order), "sampled_mesh": [n_sample, n_sample]},
            "cpu_baseline": {"value": round(v, 5), "unit": "Mcell-stage/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 5), "unit": "Mcell-stage/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
