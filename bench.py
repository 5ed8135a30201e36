#!/usr/bin/env python3
"""Benchmark of the patchy solve on the 1025^2 workload.

Workload (one "step"): the patchy decomposition on a 1025x1025 grid of [-1,1]^2,
speed c(x) = 1 + 0.5 sin(2 pi x1) sin(2 pi x2), target disc |x| <= 0.1, 32 unit
controls, lambda = 1, h = dx, coarse grid 129^2, 16 boundary sectors; one patchy
solve for each sigma in {0, 0.02, 0.1}: coarse solve -> u_hat, a*, labels, band
ordering -> band-ordered FP32 passes -> FP64 sup-residual <= 1e-6 (FP64 polish
passes when needed).  Inputs are synthetic closed-form fields (no dataset).

Metric: node-control updates per second of the whole job (every scheme
evaluation the solves perform: coarse sweeps, fine passes, FP64 residuals), with
the time to FP64 residual 1e-6 of the patchy path and of plain full-grid FP32
Jacobi value iteration (the comparator) on the same GPU reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload patchy1025|large4097|batched512]

--workload large4097 runs the 4097^2 workload instead (random Fourier speed,
six rectangular obstacles, 64 controls, sigma = 0.01, 64 patches; one patchy
solve per step, the plain Jacobi comparator timed once).  --workload
batched512 solves 512 independent instances (n 65..513) as one batch per step
against the batched plain Jacobi comparator.

N > 1 runs under torchrun, one rank per GPU; every rank solves the same
workload (independent replicas, weak scaling) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import hjb_inputs as hi  # noqa: E402

SIGMAS = (0.0, 0.02, 0.1)
N_FINE, N_COARSE, N_PATCH = 1025, 129, 16
# FP32 pass tolerance a quarter of the FP64 residual target: the FP32 stop
# (sup-increment of the last tile visits) then leaves the FP64 residual below
# the target without extra phases
TOL32, TOL64, TOL_C = 2.5e-7, 1e-6, 1e-6
METRIC = "time to 1e-6 residual vs plain GPU value iteration; node·control updates/s"
UNIT = "node·control updates/s"
SOLVER_KW = dict(schedule=0, tile_shape=-1, tile_waves=0, tile_period=2, local_sweeps=1)
BATCH_COUNT = 512
# DRAM bytes (read + write) per launch of the warp-tile kernel on the 1025^2
# workload, mean of the three launches of a step, from one ncu capture of this
# kernel (dram__bytes_read.sum + dram__bytes_write.sum); None for the other
# workloads (not captured)
WTILES_DRAM_BYTES_1025 = 14.22e6


def flops_per_node_control(sigma: float) -> int:
    """FP32 operations of one node-control update as written in the kernel
    (FMA = 2): foot 6; per axis cell 4 (clamp 2, floor, fraction); per bilinear
    point 11 (3 differences, 2 relative offsets, 3 FMA); self weights; the two
    FMAs of N and D; the cross-multiplied comparison 2.  sigma > 0: 6 axis cells,
    4 points; sigma = 0: 2 axis cells, 1 point."""
    if sigma > 0:
        return 6 + 6 * 4 + 4 * 11 + 3 + 7 + 4 + 2
    return 6 + 2 * 4 + 11 + 1 + 4 + 2


def gathers_per_node_control(sigma: float) -> int:
    return 16 if sigma > 0 else 4


# ---------------------------------------------------------------- distributed

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value: float, ws: int, device=None) -> float:
    """Max over ranks (the timing rule: the slowest rank sets the job time)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, ws: int, device=None) -> float:
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), samples=len(sm))
        out["reasons"] = sorted(reasons)
        return out


# ---------------------------------------------------------------- workload

WORKLOAD = "patchy1025"
WORKLOAD_DESC = {
    "patchy1025": "patchy 1025x1025, c=1+0.5sin(2pi x1)sin(2pi x2), disc |x|<=0.1, "
                  "32 controls, lambda=1, h=dx, coarse 129x129, 16 patches, "
                  "sigma in {0,0.02,0.1}, FP32 passes + FP64 residual <= 1e-6",
    "large4097": "large 4097x4097, random Fourier speed in [0.2,1.8], 6 rectangular "
                 "obstacles (speed 0), disc |x|<=0.1, 64 controls, sigma=0.01, lambda=1, "
                 "h=dx, coarse 129x129, 64 patches, FP32 passes + FP64 residual <= 1e-6",
}


def workload_config(insts, ws):
    """The `config` of a patchy1025 / large4097 line (both arms)."""
    return {
        "workload": WORKLOAD_DESC[WORKLOAD],
        "n": N_FINE, "coarse_n": N_COARSE, "n_patches": insts[0].n_patches,
        "n_controls": insts[0].n_controls,
        "sigmas": [i.sigma for i in insts], "tol32": TOL32, "tol64_residual": TOL64,
        "solver": SOLVER_KW,
        "l2": ("flushed between timed steps (256 MiB write); working set < L2"
               if WORKLOAD == "patchy1025" else
               "flushed between timed steps (256 MiB write); working set > L2"),
        "parallelism": f"replicas x{ws}",
    }


def batched_config(insts, n_free, ws):
    """The `config` of a batched512 line (both arms; the GPU arm adds its autotune)."""
    return {
        "workload": f"batched {BATCH_COUNT} instances, n=8k+1 in 65..513, random Fourier speed "
                    "in [0.2,1.8], 1-3 discs r 0.05-0.15, sigma~U[0,0.1], lambda~U[0.5,2], "
                    "32 controls, 4-16 patches, coarse (n-1)/4+1, FP32 passes + FP64 residual <= 1e-6",
        "instances": BATCH_COUNT, "nodes": sum(i.n * i.n for i in insts), "free_nodes": n_free,
        "tol32": TOL32, "tol64_residual": TOL64,
        "l2": "flushed between timed steps (256 MiB write); working set > L2",
        "parallelism": f"replicas x{ws}",
    }


def make_instances():
    """(label, instance) pairs of one step."""
    if WORKLOAD == "large4097":
        return [("0.01", hi.large_instance(n=N_FINE, coarse_n=N_COARSE))]
    return [(f"{s}", hi.patchy_1025(s, n=N_FINE, coarse_n=N_COARSE, n_patches=N_PATCH))
            for s in SIGMAS]


def set_size(n: int, coarse_n: int):
    """Smaller grids of the same workload (profiling captures)."""
    global N_FINE, N_COARSE
    N_FINE, N_COARSE = n, coarse_n


def flush_l2(torch, buf):
    buf.add_(1.0)          # writes 256 MiB > 129 MB of L2


def run_patchy(P, n_free):
    """One patchy solve on a created problem; returns (stats, node-control updates):
    coarse sweeps + fine passes + every FP64 residual evaluation."""
    c = P.coarse_solve(tol_c=TOL_C)
    b = P.build_patches()
    s = P.solve_patches(tol32=TOL32, tol64=TOL64)
    nc = c["node_control_updates"] + s["node_control_updates"]
    nc += s["residual_evals"] * n_free * P.n_controls
    return (c, b, s), nc


def ours(args, ws, rank, local):
    import torch
    from paper_1502_01629_gb300 import Problem, kernel_launches

    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    stream = torch.cuda.current_stream()
    labeled = make_instances()
    labels = [lb for lb, _ in labeled]
    insts = [inst for _, inst in labeled]
    n_free = [int((i.mask == 0).sum()) for i in insts]
    probs = [Problem.from_instance(inst, stream=stream, **SOLVER_KW) for inst in insts]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)

    def step(record=None):
        total_nc = 0
        per = []
        for P, sig, nf in zip(probs, labels, n_free):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            stats, nc = run_patchy(P, nf)
            ev1.record(stream)
            per.append((sig, ev0, ev1, stats, nc))
            total_nc += nc
        return per, total_nc

    for _ in range(args.warmup):
        step()
        flush_l2(torch, flush)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()

    launches0 = kernel_launches()
    step_ms, total_nc, by_sigma = [], 0, {s: [] for s in labels}
    last_stats = {}
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush_l2(torch, flush)
            per, nc = step()
            torch.cuda.synchronize()
            ms = 0.0
            for sig, e0, e1, stats, _ in per:
                t = e0.elapsed_time(e1)
                by_sigma[sig].append(t)
                last_stats[sig] = stats
                ms += t
            step_ms.append(ms)
            total_nc += nc
    torch.cuda.synchronize()
    launches = kernel_launches() - launches0
    barrier(ws)
    clocks = clk.summary()

    time_s = sum(step_ms) / 1e3
    time_s_max = reduce_max(time_s, ws, device)
    nc_all = reduce_sum(float(total_nc), ws, device)
    value = nc_all / time_s_max

    # ---- plain full-grid FP32 Jacobi comparator (same GPU, same tolerances)
    plain = {}
    for P, sig in zip(probs, labels):
        ts = []
        # one untimed run first, except on the large grid (a run of seconds)
        warm_runs = 0 if WORKLOAD == "large4097" else 1
        for r in range(warm_runs + max(1, args.plain_reps)):
            flush_l2(torch, flush)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = P.solve_full(precision=32, tol=TOL32, tol64=TOL64)
            e1.record(stream)
            torch.cuda.synchronize()
            if r >= warm_runs:
                ts.append(e0.elapsed_time(e1))
        plain[sig] = dict(ms=statistics.median(ts), sweeps=st["sweeps"],
                          fp64_sweeps=st["fp64_passes"], residual=st["residual"],
                          node_control_updates=st["node_control_updates"])

    # ---- dominant kernel: the band-wave FP32 passes (stage 0 of solve_patches)
    wave_ms, wave_flops = 0.0, 0.0
    for sig, inst in zip(labels, insts):
        c, b, s = last_stats[sig]
        wave_ms += s["ms_stage"][0]
        nodes32 = s["node_updates"] - s["fp64_node_updates"]
        wave_flops += nodes32 * inst.n_controls * flops_per_node_control(inst.sigma)
    peaks = load_peaks()
    fp32_peak = 152 * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
    achieved = wave_flops / (wave_ms / 1e3) / 1e12 if wave_ms > 0 else 0.0

    # ---- end to end through the C ABI with host buffers
    e2e_ms = []
    insts_host = insts if args.e2e_reps > 0 else []
    h2d = sum(i.speed.nbytes + i.mask.nbytes + i.sector.nbytes + i.controls.nbytes
              for i in insts_host)
    d2h = sum(i.n * i.n * 8 for i in insts_host)
    e2e_nc = 0
    for r in range(args.e2e_reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nc_r = 0
        for inst, nf in zip(insts_host, n_free):
            with Problem.from_instance(inst, stream=stream, **SOLVER_KW) as P:
                _, nc = run_patchy(P, nf)
                P.get_value()
                nc_r += nc
        torch.cuda.synchronize()
        if r > 0:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            e2e_nc += nc_r
    e2e_value = e2e_nc / (sum(e2e_ms) / 1e3) if e2e_ms else None

    if rank != 0:
        return None
    patchy_ms = {s: statistics.median(v) for s, v in by_sigma.items()}
    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": sum(step_ms) / len(step_ms),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": workload_config(insts, ws),
        "time_to_1e-6_ms": {
            "patchy": {str(s): patchy_ms[s] for s in labels},
            "plain_jacobi_fp32": {str(s): plain[s]["ms"] for s in labels},
            "speedup_vs_plain": {str(s): plain[s]["ms"] / patchy_ms[s] for s in labels},
        },
        "solver_stats": {
            str(s): {
                "coarse_sweeps": last_stats[s][0]["sweeps"],
                "n_bands": last_stats[s][1]["sweeps"],
                "fp32_passes": last_stats[s][2]["fp32_passes"],
                "fp64_passes": last_stats[s][2]["fp64_passes"],
                "residual": last_stats[s][2]["residual"],
                "ms_coarse": last_stats[s][0]["ms_total"],
                "ms_build": last_stats[s][1]["ms_total"],
                "ms_fp32_passes": last_stats[s][2]["ms_stage"][0],
                "ms_fp64": last_stats[s][2]["ms_stage"][1] + last_stats[s][2]["ms_stage"][2],
                "plain_sweeps": plain[s]["sweeps"],
                "plain_fp64_sweeps": plain[s]["fp64_sweeps"],
                "plain_residual": plain[s]["residual"],
            } for s in labels},
        "roofline": {
            "kernel": "k_wtiles<float> (warp-tile pipelined FP32 passes)",
            "bound": "alu",
            "achieved": achieved,
            "peak": fp32_peak,
            "unit": "TFLOP/s",
            "frac": achieved / fp32_peak,
            "traffic": WTILES_DRAM_BYTES_1025 if (WORKLOAD == "patchy1025" and N_FINE == 1025) else None,
            "traffic_unit": "bytes per launch (ncu dram read + write)",
            "peak_source": "152 SMs x 128 FP32 lanes x 2 x sm_max_mhz (MEASURED_PEAKS.json)",
        },
        "e2e": {"value": e2e_value, "unit": UNIT,
                "ms_per_step": statistics.median(e2e_ms) if e2e_ms else None,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds,
                                           insts[1] if len(insts) > 1 else insts[0])
    return out


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    d = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "source": "fallback"}
    if os.path.exists(p):
        d.update(json.load(open(p)))
        d["source"] = "measured"
    return d


# ------------------------------------------------------------- CPU oracle leg

def ours_batched(args, ws, rank, local):
    """The many-instance workload: 512 independent problems (n = 8k + 1 in
    65..513, random Fourier speeds, 1-3 target discs, sigma ~ U[0, 0.1], lambda
    ~ U[0.5, 2], 32 controls, 4-16 patches) solved as one batch; the plain
    comparator is the batched full-grid FP32 Jacobi on the same GPU."""
    import torch
    from paper_1502_01629_gb300 import Batch, kernel_launches

    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    stream = torch.cuda.current_stream()
    insts = [hi.batched_instance(1000 + k) for k in range(BATCH_COUNT)]
    n_free = sum(int((i.mask == 0).sum()) for i in insts)
    B = Batch.from_instances(insts, stream=stream)
    tune = B.autotune(tol_c=TOL_C, tol32=TOL32)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)

    def solve():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, res = B.solve(tol_c=TOL_C, tol32=TOL32, tol64=TOL64)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), st, res

    for _ in range(args.warmup):
        solve()
        flush_l2(torch, flush)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    launches0 = kernel_launches()
    step_ms, total_nc = [], 0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush_l2(torch, flush)
            ms, st, res = solve()
            step_ms.append(ms)
            total_nc += st["node_control_updates"]
    launches = kernel_launches() - launches0
    barrier(ws)
    clocks = clk.summary()
    time_s_max = reduce_max(sum(step_ms) / 1e3, ws, device)
    value = reduce_sum(float(total_nc), ws, device) / time_s_max
    # plain batched Jacobi comparator (seconds: one untimed start-up is not needed)
    plain_ms = []
    for _ in range(max(1, args.plain_reps)):
        flush_l2(torch, flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pst, pres = B.solve_full(tol32=TOL32, tol64=TOL64)
        e1.record(stream)
        torch.cuda.synchronize()
        plain_ms.append(e0.elapsed_time(e1))
    # dominant kernel: the warp-tile FP32 passes
    nodes32 = st["node_updates"] - st["fp64_node_updates"]
    # every instance takes the sigma > 0 path of the kernel
    sig_nodes = nodes32 * 32 * flops_per_node_control(0.05)
    peaks = load_peaks()
    fp32_peak = 152 * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
    achieved = sig_nodes / (st["ms_stage"][0] / 1e3) / 1e12
    # end to end through the C ABI with host buffers: create (H2D), solve, get_value (D2H)
    e2e_ms, e2e_nc = [], 0
    h2d = sum(i.speed.nbytes + i.mask.nbytes + i.sector.nbytes for i in insts) + insts[0].controls.nbytes
    d2h = sum(i.n * i.n * 8 for i in insts)
    for r in range(args.e2e_reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with Batch.from_instances(insts, stream=stream, tile_shape=tune["tile_shape"],
                                  tile_waves=tune["tile_waves"]) as BB:
            est, _ = BB.solve(tol_c=TOL_C, tol32=TOL32, tol64=TOL64)
            for k in range(len(insts)):
                BB.get_value(k)
        torch.cuda.synchronize()
        if r > 0:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            e2e_nc += est["node_control_updates"]
    e2e_value = e2e_nc / (sum(e2e_ms) / 1e3) if e2e_ms else None
    B.close()
    if rank != 0:
        return None
    patchy = statistics.median(step_ms)
    plain = statistics.median(plain_ms)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(step_ms) / len(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": dict(batched_config(insts, n_free, ws), autotune=tune),
        "time_to_1e-6_ms": {"patchy_batch": patchy, "plain_jacobi_fp32_batch": plain,
                            "speedup_vs_plain": plain / patchy},
        "solver_stats": {"steps": st["fp32_passes"], "node_updates": st["node_updates"],
                         "fp64_node_updates": st["fp64_node_updates"], "residual_max": float(res.max()),
                         "ms_fp32_passes": st["ms_stage"][0], "ms_residuals": st["ms_stage"][1],
                         "ms_fp64": st["ms_stage"][2], "ms_coarse": st["ms_stage"][3],
                         "ms_precompute": st["ms_stage"][4], "plain_sweeps": pst["sweeps"],
                         "plain_residual_max": float(pres.max())},
        "roofline": {"kernel": "k_wtiles<float> (warp-tile FP32 passes, all instances)", "bound": "alu",
                     "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": None,
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 x sm_max_mhz (MEASURED_PEAKS.json)"},
        "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_step": statistics.median(e2e_ms) if e2e_ms else None,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        big = max(insts, key=lambda i: i.n)
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds, big)
    return out


def cpu_baseline(seconds: float, inst=None) -> dict:
    """The FP64 oracle as it stands (single-threaded Gauss-Seidel updates of the
    modified scheme) on a bounded sample of the workload: repeated Gauss-Seidel
    passes over the first rows of the grid (at most 2^20 nodes, from u = 0), as
    many as fit in about `seconds` seconds."""
    import oracle
    if inst is None:
        inst = hi.patchy_1025(0.02, n=N_FINE, coarse_n=N_COARSE, n_patches=N_PATCH)
    O = oracle.Problem.from_instance(inst)
    u = O.fix_nonfree(np.zeros(O.N))
    rows = np.arange(0, min(O.N, 1 << 20), dtype=np.int64)
    nodes = int((inst.mask[rows] == 0).sum())
    passes = 0
    t0 = time.perf_counter()
    while True:
        O.sweep_gs(u, 3, rows)
        passes += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": nodes * inst.n_controls * passes / dt, "unit": UNIT, "cores": 1,
            "kind": "oracle",
            "sample": f"{passes} Gauss-Seidel pass(es) of the FP64 oracle over the first "
                      f"{rows.size} nodes of {inst.name} ({nodes} free nodes x "
                      f"{inst.n_controls} controls), {dt:.1f} s"}


def reference(args, ws, rank, local):
    """Reference arm: the FP64 oracle on the host cores, one bounded sample of the
    selected workload per step (Gauss-Seidel updates of a block of nodes)."""
    if rank != 0:
        return None
    import oracle
    if WORKLOAD == "batched512":
        insts = [hi.batched_instance(1000 + k) for k in range(BATCH_COUNT)]
        n_free = sum(int((i.mask == 0).sum()) for i in insts)
        config = batched_config(insts, n_free, ws)
        # step k: one full sweep of instance k (about 0.1-0.7 s each)
        plan = [(insts[k % BATCH_COUNT], None) for k in range(args.warmup + args.steps)]
        what = "a full Gauss-Seidel sweep of one instance per step (instances 0, 1, ...)"
    else:
        insts = [inst for _, inst in make_instances()]
        config = workload_config(insts, ws)
        frac = 8 if WORKLOAD == "patchy1025" else 64
        # step k: the first 1/frac of the nodes of instance k mod (number of instances)
        plan = [(insts[k % len(insts)], frac) for k in range(args.warmup + args.steps)]
        what = (f"each step: Gauss-Seidel update of the first 1/{frac} of the nodes of one "
                f"instance (sigma cycling through {[i.sigma for i in insts]})")
    problems, values = {}, {}
    nodes = 0
    dt = 0.0
    for k, (inst, frac) in enumerate(plan):
        key = id(inst)
        if key not in problems:
            O = oracle.Problem.from_instance(inst)
            problems[key] = O
            values[key] = O.fix_nonfree(np.zeros(O.N))
        O, u = problems[key], values[key]
        rows = np.arange(0, O.N // frac if frac else O.N, dtype=np.int64)
        t0 = time.perf_counter()
        O.sweep_gs(u, 3, rows)
        if k >= args.warmup:
            dt += time.perf_counter() - t0
            nodes += int((inst.mask[rows] == 0).sum()) * inst.n_controls
    val = nodes / dt if dt > 0 else 0.0
    sample = f"{what}, FP64 oracle, 1 core"
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config,
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--plain-reps", type=int, default=2)
    ap.add_argument("--e2e-reps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=("patchy1025", "large4097", "batched512"),
                    default="patchy1025",
                    help="patchy1025: the 1025^2 three-sigma workload (default); large4097: "
                         "the 4097^2 64-control workload with obstacles; batched512: 512 "
                         "independent instances of 65^2..513^2 solved as one batch")
    ap.add_argument("--n", type=int, default=0, help="fine grid size (profiling only)")
    ap.add_argument("--coarse-n", type=int, default=N_COARSE)
    args = ap.parse_args(argv)
    global WORKLOAD
    WORKLOAD = args.workload
    n_default = 4097 if WORKLOAD == "large4097" else N_FINE
    set_size(args.n or n_default, args.coarse_n)
    if args.warmup < 3 and args.impl == "ours":
        print("bench.py: --warmup must be >= 3", file=sys.stderr)
    ws, rank, local = dist_env()
    if args.impl == "reference":
        out = reference(args, ws, rank, local)
    elif WORKLOAD == "batched512":
        out = ours_batched(args, ws, rank, local)
    else:
        out = ours(args, ws, rank, local)
    if out is not None:
        print(json.dumps(out), flush=True)
    if ws > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
