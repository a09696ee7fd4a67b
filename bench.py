#!/usr/bin/env python
"""Throughput of the ASE-DFF compact gas-kinetic S2O4 step on GB300.

Workload (one "step" = one full two-stage S2O4 step, CFL time step computed
on the device, of the whole mesh): 2-D Euler, gamma 1.4, periodic [0,10]^2,
2048^2 cells, isentropic vortex of strength 5 (background rho = u = v = p = 1),
ninth order ASE-DFF(9,7,5,3), CFL 0.5, tau = 0.  Synthetic, seeded-free
(deterministic) input generated by ``paper_2508_13705_gb300.inputs``.

Metric: Mcell-stage/s = cells x 2 stages x steps / device time.  The headline
``value`` is the FP32-bulk form; the plain FP64 form is measured on the same
mesh and reported under ``fp64_plain``; ``accuracy`` compares the two forms'
L1 density error at t = 10 (one period, exact solution = initial data) on a
256^2 mesh.  ``--impl reference`` times the FP64 CPU oracle instead.
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

FP32_PEAK_LANES = 128       # FP32 lanes per SM (Blackwell)
FP64_NOMINAL_TFLOPS = 1.25  # GB300 nominal FP64 rate (non-tensor), profiling recipe
HBM_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")

# Per cell, per launch of each kernel of a stage (2-D, order 9, tau = 0): the
# FP operations executed in the bulk precision (FADD + FMUL + 2 FFMA, or the
# FP64 counterparts in the plain form), the FP64 operations of the FP32-bulk
# form, and the DRAM bytes read + written.  These are the operations the
# kernels execute, not a count of the method's textbook form: algebra that
# removes work (Gram-matrix moments, skipped zero taps) lowers them.  Counted
# by ncu (one launch each, --clock-control none) on the 1024^2 vortex; every
# kernel does the same work per cell at any mesh size (one thread per cell line
# or face point), so a launch on n^2 cells processes n^2 times these.  The
# flux kernel's operations per face Gauss point are these over 2 m (n + 1) / n
# points per cell.
KERNEL_COUNTS = {
    ("fp32", 9): {"s1_lines": (612.8, 24.1, 227.5), "s1_normal": (3638.2, 0.0, 1010.4),
                  "s1_flux": (19284.7, 0.0, 1320.4), "s1_update": (544.0, 58.0, 933.9),
                  "s2_lines": (612.8, 24.1, 228.0), "s2_normal": (3638.2, 0.0, 1009.6),
                  "s2_flux": (18329.9, 0.0, 1015.3), "s2_update": (336.0, 24.0, 626.9)},
    ("fp64", 9): {"s1_lines": (637.6, 637.6, 448.5), "s1_normal": (3679.6, 3679.6, 2092.0),
                  "s1_flux": (21492.8, 21492.8, 2760.3), "s1_update": (506.0, 506.0, 1752.1),
                  "s2_lines": (637.6, 637.6, 448.8), "s2_normal": (3679.6, 3679.6, 2088.9),
                  "s2_flux": (20275.8, 20275.8, 2191.5), "s2_update": (312.0, 312.0, 1158.1)},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--order", type=int, default=9)
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-config3", action="store_true")
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


def max_over_ranks(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


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
                                       "--format=csv,noheader,nounits", "-lms", "200"],
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


def vortex_inputs(n, order, nq=4):
    from paper_2508_13705_gb300 import inputs
    return inputs.cell_state_2d(inputs.vortex_prim(), n, n, (0.0, 10.0, 0.0, 10.0), order, nq=nq)


def peaks():
    try:
        return json.load(open(HBM_PEAKS))
    except (OSError, ValueError):
        return {}


def gpu_peak_tflops(precision, sm_count, mhz):
    if precision == "fp32":
        return sm_count * FP32_PEAK_LANES * 2 * mhz * 1e6 / 1e12
    return FP64_NOMINAL_TFLOPS * mhz / 2070.0


def run_gpu_form(torch, cgks, st, n, order, precision, steps, warmup, stream):
    s = cgks.Solver(2, order, n, n, extent=(0.0, 10.0, 0.0, 10.0), precision=precision,
                    stream=stream.cuda_stream)
    s.set_state(*st)
    s.advance(warmup, 0.0)
    s.sync()
    return s


def cpu_oracle_rate(order, n_sample, steps):
    """FP64 CPU oracle on a bounded sample of the workload (same problem, smaller mesh)."""
    import oracle
    oracle.build()
    st = vortex_inputs(n_sample, order, nq=4)
    o = oracle.Oracle(2, order, n_sample, n_sample, extent=(0.0, 10.0, 0.0, 10.0))
    o.set_state(*st)
    o.step()  # first call loads the library
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step()
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return n_sample * n_sample * 2 * steps / el / 1e6, cores, el


def main():
    a = parse()
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

    # ---------------- FP32-bulk form (headline)
    s32 = run_gpu_form(torch, cgks, st, n, order, cgks.FP32_BULK, a.steps, a.warmup, stream)
    tuned32 = s32.autotune()
    s32.advance(1, 0.0)
    s32.sync()
    kps = s32.kernels_per_step()
    clk = ClockSampler(local)
    clk.start()
    barrier(pg)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed steps
    e0.record(stream)
    s32.advance(a.steps, 0.0)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier(pg)
    ms32 = max_over_ranks(pg, e0.elapsed_time(e1))
    clocks = clk.stop()
    _, rc32, _ = s32.sync(raise_on_error=False)
    dt = s32.compute_dt()
    prof32 = s32.profile_step(dt)

    # ---------------- FP64 plain form, same mesh
    k64 = max(2, a.steps // 5)
    s64 = run_gpu_form(torch, cgks, st, n, order, cgks.FP64, k64, 1, stream)
    tuned64 = s64.autotune()
    barrier(pg)
    torch.cuda.synchronize()
    e0.record(stream)
    s64.advance(k64, 0.0)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    ms64 = max_over_ranks(pg, e0.elapsed_time(e1))
    _, rc64, _ = s64.sync(raise_on_error=False)
    prof64 = s64.profile_step(s64.compute_dt())
    s64.close()

    # ---------------- end to end: host (pinned) state in, step, state out
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

    value = world * cells * 2 * a.steps / (ms32 / 1e3) / 1e6
    v64 = world * cells * 2 * k64 / (ms64 / 1e3) / 1e6
    e2e_v = world * cells * 2 * k_e2e / e2e_s / 1e6

    # ---------------- roofline of the dominant kernel (plain ALU arithmetic)
    props = torch.cuda.get_device_properties(local)
    sm_count = props.multi_processor_count
    mhz = clocks.get("sm_max_mhz") or 2070.0
    names_k = {0: "lines", 1: "normal", 2: "flux", 3: "update", 4: "dt"}

    def roof(prof, precision):
        """Achieved FP rate of every kernel of the step against the FP pipe peak;
        the headline entry is the kernel with the largest share of the step."""
        counts = KERNEL_COUNTS.get((precision, order), {})
        peak = gpu_peak_tflops(precision, sm_count, mhz)
        hbm = peaks().get("hbm_gbs")
        total = sum(x[1] for x in prof)
        kms = {("s%d_" % (k // 10) if k >= 10 else "") + names_k[k % 10]: v for k, v in prof}
        per = {}
        for name, ms in kms.items():
            if name not in counts:
                continue
            fl, _, by = counts[name]
            ach = fl * cells / (ms / 1e3) / 1e12
            gbs = by * cells / (ms / 1e3) / 1e9
            per[name] = {"ms": round(ms, 4), "achieved_tflops": round(ach, 3), "frac": round(ach / peak, 4),
                         "dram_gbs": round(gbs, 1), "dram_frac": round(gbs / hbm, 4) if hbm else None}
        top = max(per, key=lambda k: per[k]["ms"]) if per else None
        fl, _, by = counts[top] if top else (None, None, None)
        ach = per[top]["achieved_tflops"] if top else None
        return {"bound": "alu", "kernel": top,
                "achieved": ach, "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": None if ach is None else ach / peak,
                "traffic": None if by is None else round(by * cells),
                "traffic_basis": "ncu dram__bytes_read.sum + dram__bytes_write.sum per cell on 1024^2, "
                                 "times the launch's cells",
                "flops_per_cell": fl,
                "share_of_step": None if top is None else kms[top] / total,
                "peak_basis": ("%d SMs x %d FP32 lanes x 2 x %.0f MHz" % (sm_count, FP32_PEAK_LANES, mhz))
                if precision == "fp32" else "nominal FP64 1.25 TFLOP/s at 2070 MHz, scaled to %.0f MHz" % mhz,
                "kernels": per,
                "kernels_ms": {k: round(v, 4) for k, v in kms.items()}}

    line = {
        "metric": "Mcell-stage/s 2D 9th-order, FP32 form vs FP64 plain at fixed L1 err; %roofline",
        "value": round(value, 3), "unit": "Mcell-stage/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(ms32 / a.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "isentropic vortex 2-D, periodic [0,10]^2, %dx%d cells, order %d, CFL 0.5, tau 0"
                               % (n, n, order), "precision": "FP32 bulk, FP64 cell averages and accumulation",
                   "global_batch": world, "mesh": [n, n], "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (state %.2f GB per replica)" % (bytes_state / 1e9)},
        "fp64_plain": {"value": round(v64, 3), "unit": "Mcell-stage/s", "steps": k64,
                       "ms_per_step": round(ms64 / k64, 4), "status": rc64,
                       "roofline": roof(prof64, "fp64")},
        "roofline": roof(prof32, "fp32"),
        "clocks": clocks,
        "e2e": {"value": round(e2e_v, 3), "unit": "Mcell-stage/s", "h2d_bytes_per_step": bytes_state,
                "d2h_bytes_per_step": bytes_state, "steps": k_e2e},
        "gpu_launches": kps * a.steps,
        "autotuned_threads": {"fp32": tuned32, "fp64": tuned64},
        "status": rc32,
        "input_gen_s": round(t_in, 2),
    }
    if rank == 0 and not a.no_accuracy:
        line["accuracy"] = accuracy(torch, cgks, order, stream)
    if rank == 0 and not a.no_batch:
        line["batch"] = batch_bench(torch, cgks, stream)
    if rank == 0 and not a.no_config3:
        line["config3"] = config3_bench(torch, cgks, stream)
    if rank == 0 and not a.no_cpu:
        rate, cores, el = cpu_oracle_rate(order, 128, 2)
        line["cpu_baseline"] = {"value": round(rate, 5), "unit": "Mcell-stage/s", "cores": cores, "kind": "oracle",
                                "sample": "2 steps of the same vortex problem on a 128^2 mesh (%.1f s)" % el}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def accuracy(torch, cgks, order, stream, meshes=(64, 128, 256), t_end=10.0):
    """L1 density error of both forms at t = 10 (one period) on several meshes;
    reports the finest mesh where the FP32-bulk error is within 10% of FP64's."""
    rows = [accuracy_one(torch, cgks, order, stream, n, t_end) for n in meshes]
    ok = [r["mesh"][0] for r in rows if r["within_10pct"]]
    return {"t": t_end, "rows": rows, "finest_mesh_within_10pct": max(ok) if ok else None}


def accuracy_one(torch, cgks, order, stream, n, t_end):
    from paper_2508_13705_gb300 import inputs
    st = inputs.vortex_2d(n, order)
    out = {"mesh": [n, n], "t": t_end}
    for name, prec in (("fp64", cgks.FP64), ("fp32", cgks.FP32_BULK)):
        s = cgks.Solver(2, order, n, n, extent=(0.0, 10.0, 0.0, 10.0), precision=prec, stream=stream.cuda_stream)
        s.set_state(*st)
        t, steps, rc = s.run_to(t_end, max_steps=20000)
        W = s.get_state()["W"]
        out["l1_" + name] = float(np.abs(W[0] - st[0][0]).mean())
        out["status_" + name] = rc
        out["steps"] = steps
        s.close()
    out["fp32_over_fp64"] = out["l1_fp32"] / out["l1_fp64"]
    out["within_10pct"] = out["fp32_over_fp64"] <= 1.10
    return out


def batch_bench(torch, cgks, stream, count=256, order=7, steps=10):
    """Config C5: 256 seeded uneven periodic meshes (sides 64-512, smooth modes
    plus a planar shock), order 7, HGKS tau.  FP32-bulk batch (one persistent
    launch per kernel, one graph per step, device CFL per instance) against
    the same instances stepped one at a time in FP64."""
    from paper_2508_13705_gb300 import inputs
    sp = inputs.batch_specs(count, seed=0)
    t0 = time.perf_counter()
    states = [inputs.batch_instance(s, order, nq=2) for s in sp]
    t_in = time.perf_counter() - t0
    nx = [s["nx"] for s in sp]
    ny = [s["ny"] for s in sp]
    ext = [(0.0, 1.0, 0.0, s["ny"] / s["nx"]) for s in sp]
    cells = sum(x * y for x, y in zip(nx, ny))
    b = cgks.Batch(order, nx, ny, ext, precision=cgks.FP32_BULK, tau_mode=cgks.TAU_HGKS, stream=stream.cuda_stream)
    for k, st in enumerate(states):
        b.set_state(k, *st)
    tuned = b.autotune()
    for _ in range(2):
        b.step(None)
    b.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
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
    # FP64, one instance at a time
    k64 = 2
    ms64 = 0.0
    for k, st in enumerate(states):
        s = cgks.Solver(2, order, nx[k], ny[k], extent=ext[k], precision=cgks.FP64, tau_mode=cgks.TAU_HGKS,
                        stream=stream.cuda_stream)
        s.set_state(*st)
        s.advance(1, 0.0)
        torch.cuda.synchronize()
        e0.record(stream)
        s.advance(k64, 0.0)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 += e0.elapsed_time(e1)
        s.close()
    return {"workload": "%d periodic instances, sides 64-512 (seed 0), Fourier modes + Mach 1.5-3 planar shock, "
                        "order %d, HGKS tau, CFL 0.5" % (count, order),
            "cells": cells, "fp32_batched": {"value": round(cells * 2 * steps / (ms32 / 1e3) / 1e6, 3),
                                             "unit": "Mcell-stage/s", "steps": steps, "status": rc,
                                             "autotuned_threads": tuned},
            "fp64_one_at_a_time": {"value": round(cells * 2 * k64 / (ms64 / 1e3) / 1e6, 3),
                                   "unit": "Mcell-stage/s", "steps": k64},
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
    reconstruction-only CPU times; (2) the full run at 500^2 to t = 0.6."""
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
    full = {}
    for prec, key in ((cgks.FP32_BULK, "fp32"), (cgks.FP64, "fp64")):
        s = solver(500, full_order, prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t, steps, rc = s.run_to(0.6, max_steps=20000)
        wall = time.perf_counter() - t0
        s.close()
        full[key] = {"steps": steps, "wall_s": round(wall, 3), "status": rc,
                     "Mcell_stage_per_s": round(500 * 500 * 2 * steps / wall / 1e6, 3)}
    return {"workload": "2-D Riemann Configuration 3 (Sec. 4.7), transmissive, HGKS tau, CFL 0.5",
            "twenty_steps": table,
            "full_run_500_t0.6_order%d" % full_order: full,
            "note": "paper times: reconstruction only, one CPU core; GPU times: whole steps incl. CFL"}


def reference_arm(a):
    """The FP64 CPU oracle, timed on the host cores, on bounded samples."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    n_sample = 96
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
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    v = n_sample * n_sample * 2 * a.steps / el / 1e6
    sample = "the %dx%d vortex problem (same physics and order as the %d^2 workload), one S2O4 step per step" % (
        n_sample, n_sample, a.n)
    line = {"impl": "reference", "metric": "Mcell-stage/s 2D 9th-order, FP32 form vs FP64 plain at fixed L1 err; %roofline",
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
