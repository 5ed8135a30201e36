#!/usr/bin/env python3
"""Benchmark: time to FP64 sup-residual 1e-6 of the patchy solve against plain
full-grid FP32 Jacobi value iteration on the same GPU, and node-control updates/s.

Default workload, one "step" (the large problem): 4097 x 4097 grid of [-1,1]^2,
random Fourier speed clipped to [0.2, 1.8] (seed 5000), six rectangular obstacles
(speed 0, held at the obstacle value), target disc |x| <= 0.1, 64 unit controls,
sigma = 0.01, lambda = 1, h = dx, coarse grid 129^2, 64 boundary sectors; one
patchy solve: coarse solve -> u_hat, a*, labels, tile waves -> FP32 passes ->
FP64 sup-residual <= 1e-6 (FP64 passes only if needed).  Inputs are synthetic
closed-form or seeded fields (no dataset).  The comparator, plain FP32 Jacobi
from u = 0 to the same FP64 residual, is timed after the timed steps.

Every result carries its error against the FP64 CPU oracle: at 4097^2 the
largest difference from the oracle's solution at a seeded sample of nodes (when
tests/golden holds it) and the certified bound r / (1 - beta) of the FP64
residual r (the scheme is a beta-contraction); the solve to the residual that
certifies the gate 1e-5 max(1, |u|) is timed too.  The same line carries the
1025^2 workload (sigma in {0, 0.02, 0.1}; every node compared with the oracle's
solution) and the 512-instance batch as extra keys.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload large4097|patchy1025|batched512] [--no-extras]

N > 1 runs under torchrun, one rank per GPU; every rank solves the same
workload (independent replicas, weak scaling) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import contextlib
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
TOL32, TOL64, TOL_C = 1.25e-7, 1e-6, 1e-6
# value gate of the FP32 results against the FP64 oracle: 1e-5 max(1, |u|)
GATE_REL = 1e-5
METRIC = "time to 1e-6 residual vs plain GPU value iteration; node·control updates/s"
UNIT = "node·control updates/s"
SOLVER_KW = dict(schedule=0, tile_shape=-1, tile_waves=0, tile_period=0, local_sweeps=0, visit=0)
BATCH_COUNT = 512
GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")
# DRAM bytes (read + write) per launch of the FP32 patch kernel, from one ncu
# capture of the current kernel (dram__bytes_read.sum + dram__bytes_write.sum;
# profiles/dram_traffic_wtiles.md), per workload: 4097^2 one launch per solve;
# 1025^2 the mean of a step's three launches; None where no capture exists
WTILES_DRAM_BYTES = {"patchy1025": 14.25e6, "large4097": 257.23e6, "batched512": None}


def ops_per_node_control(sigma: float) -> int:
    """Algorithmic FP32 operations of one node-control update of eq. SLscheme3
    (FMA = 2): the foot (2 FMAs), one floor/fraction pair per distinct axis
    coordinate (six with diffusion: the +-e1 points share a row, the +-e2 points a
    column; two without), 24 for four bilinear interpolations (6 each), about 12 for
    the self weights and Lambda0, 6 for the sums and 3 for the cross-multiplied
    minimum: about 60 with sigma > 0; one bilinear, two axis pairs and the same
    bookkeeping, about 18, with sigma = 0."""
    return 60 if sigma > 0 else 18


def gathers_per_node_control(sigma: float) -> int:
    """Four-byte shared-memory gathers of one node-control update: four Q1
    vertices per Markov-chain point, four points with diffusion, one without."""
    return 16 if sigma > 0 else 4


def ops_as_written(sigma: float) -> int:
    """FP32 operations of one node-control update as the kernel writes them (FMA =
    2; a side figure): foot 6; per axis cell 4 (clamp 2, floor, fraction); per
    bilinear point 11 (3 differences, 2 relative offsets, 3 FMA); self weights;
    the two FMAs of N and D; the comparison 2."""
    if sigma > 0:
        return 6 + 6 * 4 + 4 * 11 + 3 + 7 + 4 + 2
    return 6 + 2 * 4 + 11 + 1 + 4 + 2


def sm_peaks(peaks: dict) -> dict:
    """On-SM peaks of the GB300 at the measured maximum SM clock: FP32 = 152 SMs x
    128 lanes x 2 (FMA) per clock; shared memory = 152 SMs x 32 four-byte words
    per clock (32 banks)."""
    mhz = peaks["sm_max_mhz"] * 1e6
    return {"fp32_tflops": 152 * 128 * 2 * mhz / 1e12, "smem_twords": 152 * 32 * mhz / 1e12}


def roofline_entry(kernel: str, parts, kernel_ms: float, peaks: dict, traffic=None) -> dict:
    """The roofline of the FP32 patch passes from (sigma, n_controls, FP32 node
    updates) parts and the kernel time: algorithmic ops and gathers per
    node-control as counted above, against the FP32 and shared-memory peaks.
    The binding resource (the larger fraction) gives `frac`."""
    pk = sm_peaks(peaks)
    t = kernel_ms / 1e3
    ops = sum(nodes * na * ops_per_node_control(sig) for sig, na, nodes in parts)
    words = sum(nodes * na * gathers_per_node_control(sig) for sig, na, nodes in parts)
    written = sum(nodes * na * ops_as_written(sig) for sig, na, nodes in parts)
    f32 = ops / t / 1e12 if t > 0 else 0.0
    lsu = words / t / 1e12 if t > 0 else 0.0
    frac_fp32 = f32 / pk["fp32_tflops"]
    frac_lsu = lsu / pk["smem_twords"]
    smem_bound = frac_lsu >= frac_fp32
    return {
        "kernel": kernel,
        "bound": "alu",
        "resource": "shared-memory gathers" if smem_bound else "FP32 pipe",
        "achieved": lsu if smem_bound else f32,
        "peak": pk["smem_twords"] if smem_bound else pk["fp32_tflops"],
        "unit": "Tword/s" if smem_bound else "TFLOP/s",
        "frac": max(frac_fp32, frac_lsu),
        "frac_fp32": frac_fp32,
        "frac_lsu": frac_lsu,
        "fp32_tflops": f32,
        "smem_twords_per_s": lsu,
        "fp32_tflops_as_written": written / t / 1e12 if t > 0 else 0.0,
        "kernel_ms": kernel_ms,
        "fp32_node_control_updates": sum(nodes * na for _, na, nodes in parts),
        "traffic": traffic,
        "traffic_unit": "bytes per launch (ncu dram read + write)",
        "peak_source": ("of measured sm_max_mhz (MEASURED_PEAKS.json): FP32 152 x 128 x 2 per clock, "
                        "shared memory 152 x 32 words per clock" if peaks.get("source") == "measured"
                        else "of fallback clock 2070 MHz"),
    }


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

WORKLOAD_DESC = {
    "patchy1025": "patchy 1025x1025, c=1+0.5sin(2pi x1)sin(2pi x2), disc |x|<=0.1, "
                  "32 controls, lambda=1, h=dx, coarse 129x129, 16 patches, "
                  "sigma in {0,0.02,0.1}, FP32 passes + FP64 residual <= 1e-6",
    "large4097": "large 4097x4097, random Fourier speed in [0.2,1.8], 6 rectangular "
                 "obstacles (speed 0), disc |x|<=0.1, 64 controls, sigma=0.01, lambda=1, "
                 "h=dx, coarse 129x129, 64 patches, FP32 passes + FP64 residual <= 1e-6",
}


def make_instances(workload: str, n: int = 0, coarse_n: int = N_COARSE):
    """(label, instance) pairs of one step of a single-problem workload."""
    if workload == "large4097":
        return [("0.01", hi.large_instance(n=n or 4097, coarse_n=coarse_n))]
    return [(f"{s}", hi.patchy_1025(s, n=n or N_FINE, coarse_n=coarse_n, n_patches=N_PATCH))
            for s in SIGMAS]


def workload_config(workload: str, insts, ws: int) -> dict:
    """The `config` of a single-problem workload (both arms)."""
    return {
        "workload": WORKLOAD_DESC[workload],
        "n": insts[0].n, "coarse_n": insts[0].coarse_n, "n_patches": insts[0].n_patches,
        "n_controls": insts[0].n_controls,
        "sigmas": [i.sigma for i in insts], "tol32": TOL32, "tol64_residual": TOL64,
        "solver": SOLVER_KW,
        "l2": ("flushed between timed steps (256 MiB write); working set < L2"
               if insts[0].n <= 1025 else
               "flushed between timed steps (256 MiB write); working set > L2"),
        "parallelism": f"replicas x{ws}",
    }


def batched_config(insts, n_free, ws) -> dict:
    """The `config` of the batched512 workload (both arms; the GPU arm adds its autotune)."""
    return {
        "workload": f"batched {BATCH_COUNT} instances, n=8k+1 in 65..513, random Fourier speed "
                    "in [0.2,1.8], 1-3 discs r 0.05-0.15, sigma~U[0,0.1], lambda~U[0.5,2], "
                    "32 controls, 4-16 patches, coarse (n-1)/4+1, FP32 passes + FP64 residual <= 1e-6",
        "instances": BATCH_COUNT, "nodes": sum(i.n * i.n for i in insts), "free_nodes": n_free,
        "tol32": TOL32, "tol64_residual": TOL64,
        "l2": "flushed between timed steps (256 MiB write); working set > L2",
        "parallelism": f"replicas x{ws}",
    }


def flush_l2(buf):
    buf.add_(1.0)          # writes 256 MiB > 129 MB of L2


def beta_of(inst) -> float:
    return 1.0 / (1.0 + inst.lam * inst.h_eff)


def certify_tol(inst) -> float:
    """The FP64 residual r whose bound r / (1 - beta) on |u - u*| meets the value
    gate 1e-5 max(1, |u|) (|u| <= h l / (1 - beta) on this problem class)."""
    umax = inst.h_eff * inst.cost / (1.0 - beta_of(inst))
    return GATE_REL * max(1.0, umax) * (1.0 - beta_of(inst)) * 0.99


def golden_name(workload: str, inst) -> str:
    if workload == "large4097":
        return f"large{inst.n}_sigma0.01"
    return f"patchy1025_sigma{inst.sigma:g}"


def load_golden(workload: str, inst):
    """The oracle's solution of this instance, written by tests/golden/make_full_size.py
    (FP64 oracle only), or None when the file is absent or of another size."""
    p = os.path.join(GOLDEN_DIR, golden_name(workload, inst) + ".npz")
    if not os.path.exists(p):
        return None
    g = dict(np.load(p))
    if int(g["n"]) != inst.n or abs(float(g["sigma"]) - inst.sigma) > 0:
        return None
    return g


def value_gate(u: np.ndarray, inst, residual: float, golden) -> dict:
    """Error of a result against the FP64 oracle: every node where the oracle's
    solution is stored, a seeded sample of nodes otherwise; with the certified
    bound r / (1 - beta) from the result's own FP64 residual r."""
    bound = residual / (1.0 - beta_of(inst))
    out = {"residual": residual, "err_bound": bound,
           "gate": GATE_REL * max(1.0, float(np.abs(u).max()))}
    if golden is not None:
        if "u32" in golden:
            ref = golden["u32"].astype(np.float64)
            out["oracle_err"] = float(np.abs(u - ref).max())
            out["compared"] = "every node (oracle solution rounded to FP32, 6e-8 relative)"
        else:
            idx = golden["idx"]
            out["oracle_err"] = float(np.abs(u[idx] - golden["u64"]).max())
            out["compared"] = f"{idx.size} seeded free nodes (oracle FP64)"
        out["oracle_residual"] = float(golden["residual"])
        out["pass"] = bool(out["oracle_err"] <= out["gate"])
    else:
        out["pass"] = bool(bound <= out["gate"])
        out["compared"] = "certified bound only (no stored oracle solution)"
    return out


def run_patchy(P, tol64=None):
    """One patchy solve on a created problem; returns (stats, node-control updates):
    coarse sweeps + fine FP32/FP64 passes (the residual evaluations are not updates)."""
    c = P.coarse_solve(tol_c=TOL_C)
    b = P.build_patches()
    s = P.solve_patches(tol32=TOL32, tol64=TOL64 if tol64 is None else tol64)
    return (c, b, s), c["node_control_updates"] + s["node_control_updates"]


def event_pair(torch, stream):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    return e0, e1


def pinned(torch, a: np.ndarray) -> np.ndarray:
    """A copy of `a` in pinned (page-locked) host memory, as a numpy view."""
    t = torch.empty(a.shape, dtype=getattr(torch, a.dtype.name), pin_memory=True)
    out = t.numpy()
    out[...] = a
    return out


def pinned_instance(torch, inst):
    """The instance with its uploaded arrays (speed, mask, sectors, controls) in
    pinned host memory: the end-to-end path's inputs, as a caller staging them
    for repeated solves would hold them."""
    import dataclasses
    return dataclasses.replace(inst, speed=pinned(torch, inst.speed), mask=pinned(torch, inst.mask),
                               sector=pinned(torch, inst.sector), controls=pinned(torch, inst.controls))


# --------------------------------------------------- single-problem workloads

def bench_single(workload: str, insts, labels, *, steps: int, warmup: int, plain_reps: int,
                 e2e_reps: int, certify: bool, ws: int, device, stream, sample_clocks: bool = True):
    """Time `steps` patchy solves of every instance (after `warmup` untimed ones),
    then the end-to-end path through the C ABI with host buffers, the value gate of
    each result, optionally the certifying solve, and the plain Jacobi comparator."""
    import torch
    from paper_1502_01629_gb300 import Problem, kernel_launches

    probs = [Problem.from_instance(inst, stream=stream, **SOLVER_KW) for inst in insts]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)

    def step():
        per, total = [], 0
        for P, lb in zip(probs, labels):
            e0, e1 = event_pair(torch, stream)
            e0.record(stream)
            stats, nc = run_patchy(P)
            e1.record(stream)
            per.append((lb, e0, e1, stats))
            total += nc
        return per, total

    for _ in range(warmup):
        step()
        flush_l2(flush)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    launches0 = kernel_launches()
    step_ms, total_nc, by_label, last = [], 0, {lb: [] for lb in labels}, {}
    clk = ClockSampler(device.index) if sample_clocks else contextlib.nullcontext()
    with clk:
        for _ in range(steps):
            flush_l2(flush)
            per, nc = step()
            torch.cuda.synchronize()
            ms = 0.0
            for lb, e0, e1, stats in per:
                t = e0.elapsed_time(e1)
                by_label[lb].append(t)
                last[lb] = stats
                ms += t
            step_ms.append(ms)
            total_nc += nc
    torch.cuda.synchronize()
    launches = kernel_launches() - launches0
    barrier(ws)
    clocks = clk.summary() if sample_clocks else None
    time_s_max = reduce_max(sum(step_ms) / 1e3, ws, device)
    value = reduce_sum(float(total_nc), ws, device) / time_s_max

    # end to end through the C ABI with host buffers in pinned memory (staged
    # once, outside the timed region): create (H2D), solve, get_value (D2H); run
    # right after the timed steps, in the same state of the GPU (before the
    # comparator's seconds of full-grid sweeps)
    e2e_ms, e2e_nc = [], 0
    h2d = sum(i.speed.nbytes + i.mask.nbytes + i.sector.nbytes + i.controls.nbytes for i in insts)
    d2h = sum(i.n * i.n * 8 for i in insts)
    host_in = [pinned_instance(torch, i) for i in insts] if e2e_reps > 0 else []
    host_out = [pinned(torch, np.zeros(i.n * i.n)) for i in host_in]
    for r in range(e2e_reps + 1 if e2e_reps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nc_r = 0
        for inst, out in zip(host_in, host_out):
            with Problem.from_instance(inst, stream=stream, **SOLVER_KW) as P:
                _, nc = run_patchy(P)
                P.get_value(out=out)
                nc_r += nc
        torch.cuda.synchronize()
        if r > 0:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            e2e_nc += nc_r

    # value gate of the last timed result of each instance (outside the timed region)
    gates = {}
    for P, lb, inst in zip(probs, labels, insts):
        gates[lb] = value_gate(P.get_value(), inst, last[lb][2]["residual"],
                               load_golden(workload, inst))

    # the solve to the residual that certifies the gate through r / (1 - beta)
    certified = {}
    if certify:
        for P, lb, inst in zip(probs, labels, insts):
            tol = certify_tol(inst)
            flush_l2(flush)
            e0, e1 = event_pair(torch, stream)
            e0.record(stream)
            (c, b, s), _ = run_patchy(P, tol64=tol)
            e1.record(stream)
            torch.cuda.synchronize()
            g = value_gate(P.get_value(), inst, s["residual"], load_golden(workload, inst))
            certified[lb] = dict(tol64_residual=tol, ms=e0.elapsed_time(e1),
                                 fp64_passes=s["fp64_passes"], **g)

    # plain full-grid FP32 Jacobi comparator (same GPU, same tolerances)
    plain = {}
    for P, lb, inst in zip(probs, labels, insts):
        ts = []
        warm_runs = 0 if inst.n > 2049 else 1    # a run of seconds needs no start-up run
        for r in range(warm_runs + plain_reps if plain_reps > 0 else 0):
            flush_l2(flush)
            e0, e1 = event_pair(torch, stream)
            e0.record(stream)
            st = P.solve_full(precision=32, tol=TOL32, tol64=TOL64)
            e1.record(stream)
            torch.cuda.synchronize()
            if r >= warm_runs:
                ts.append(e0.elapsed_time(e1))
        if not ts:         # --plain-reps 0 (profiling): no comparator
            plain[lb] = dict(ms=float("nan"), sweeps=0, fp64_sweeps=0)
            continue
        plain[lb] = dict(ms=statistics.median(ts), sweeps=st["sweeps"], fp64_sweeps=st["fp64_passes"],
                         **value_gate(P.get_value(), inst, st["residual"],
                                      load_golden(workload, inst)))

    # the FP32 patch kernel: stage 0 of solve_patches (CUDA events on the solver's stream)
    parts, kernel_ms = [], 0.0
    for lb, inst in zip(labels, insts):
        s = last[lb][2]
        kernel_ms += s["ms_stage"][0]
        parts.append((inst.sigma, inst.n_controls, s["node_updates"] - s["fp64_node_updates"]))

    for P in probs:
        P.close()
    patchy_ms = {lb: statistics.median(v) for lb, v in by_label.items()}
    return dict(
        value=value, step_ms=step_ms, launches=launches, clocks=clocks,
        time_to={"patchy": patchy_ms, "plain_jacobi_fp32": {lb: plain[lb]["ms"] for lb in labels},
                 "speedup_vs_plain": {lb: plain[lb]["ms"] / patchy_ms[lb] for lb in labels}},
        gates=gates, certified=certified, plain=plain, last=last, parts=parts, kernel_ms=kernel_ms,
        e2e=dict(value=e2e_nc / (sum(e2e_ms) / 1e3) if e2e_ms else None, unit=UNIT,
                 ms_per_step=statistics.median(e2e_ms) if e2e_ms else None,
                 h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h))


def single_summary(workload: str, insts, labels, R: dict, peaks: dict) -> dict:
    """Per-workload keys of a single-problem result (the headline line or an extra)."""
    out = {
        "time_to_1e-6_ms": {k: {str(lb): v for lb, v in d.items()} for k, d in R["time_to"].items()},
        "value_gate": {
            "rule": "max |u - u_oracle| <= 1e-5 max(1, |u|) (FP32 gate); oracle = FP64 CPU "
                    "Gauss-Seidel to sup-increment 1e-13 (tests/golden/make_full_size.py)",
            "patchy": R["gates"], "plain_jacobi_fp32": {lb: {k: v for k, v in p.items()
                                                            if k not in ("ms", "sweeps", "fp64_sweeps")}
                                                       for lb, p in R["plain"].items()}},
        "solver_stats": {
            str(lb): {
                "coarse_sweeps": R["last"][lb][0]["sweeps"],
                "fp32_passes": R["last"][lb][2]["fp32_passes"],
                "fp64_passes": R["last"][lb][2]["fp64_passes"],
                "residual": R["last"][lb][2]["residual"],
                "ms_coarse": R["last"][lb][0]["ms_total"],
                "ms_build": R["last"][lb][1]["ms_total"],
                "ms_fp32_passes": R["last"][lb][2]["ms_stage"][0],
                "ms_fp64": R["last"][lb][2]["ms_stage"][1] + R["last"][lb][2]["ms_stage"][2],
                "plain_sweeps": R["plain"][lb]["sweeps"],
                "plain_fp64_sweeps": R["plain"][lb]["fp64_sweeps"],
            } for lb in labels},
        "roofline": roofline_entry("k_wtiles<float> (FP32 patch passes)", R["parts"], R["kernel_ms"],
                                   peaks, WTILES_DRAM_BYTES.get(workload)),
        "e2e": R["e2e"],
    }
    if R["certified"]:
        out["time_to_certified_ms"] = {str(lb): c["ms"] for lb, c in R["certified"].items()}
        out["value_gate"]["certified_solve"] = R["certified"]
    return out


# ------------------------------------------------------------ the batch

def bench_batched(*, steps: int, warmup: int, plain_reps: int, e2e_reps: int, ws: int, device,
                  stream, peaks: dict, sample_clocks: bool = True, certify: bool = True):
    """The many-instance workload: 512 independent problems (n = 8k + 1 in 65..513,
    random Fourier speeds, 1-3 target discs, sigma ~ U[0, 0.1], lambda ~ U[0.5, 2],
    32 controls, 4-16 patches) solved as one batch per step; the comparator is the
    batched full-grid FP32 Jacobi on the same GPU."""
    import torch
    from paper_1502_01629_gb300 import Batch, kernel_launches

    insts = [hi.batched_instance(1000 + k) for k in range(BATCH_COUNT)]
    n_free = sum(int((i.mask == 0).sum()) for i in insts)
    B = Batch.from_instances(insts, stream=stream)
    tune = B.autotune(tol_c=TOL_C, tol32=TOL32)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)
    betas = np.array([beta_of(i) for i in insts])

    def solve():
        e0, e1 = event_pair(torch, stream)
        e0.record(stream)
        st, res = B.solve(tol_c=TOL_C, tol32=TOL32, tol64=TOL64)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), st, res

    for _ in range(warmup):
        solve()
        flush_l2(flush)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    launches0 = kernel_launches()
    step_ms, total_nc = [], 0
    clk = ClockSampler(device.index) if sample_clocks else contextlib.nullcontext()
    with clk:
        for _ in range(steps):
            flush_l2(flush)
            ms, st, res = solve()
            step_ms.append(ms)
            total_nc += st["node_control_updates"]
    launches = kernel_launches() - launches0
    barrier(ws)
    clocks = clk.summary() if sample_clocks else None
    time_s_max = reduce_max(sum(step_ms) / 1e3, ws, device)
    value = reduce_sum(float(total_nc), ws, device) / time_s_max
    # end to end through the C ABI with host buffers in pinned memory (staged
    # once, outside the timed region): create (H2D), solve, values (D2H); run
    # right after the timed steps, in the same state of the GPU
    e2e_ms, e2e_nc = [], 0
    h2d = sum(i.speed.nbytes + i.mask.nbytes + i.sector.nbytes for i in insts) + insts[0].controls.nbytes
    d2h = sum(i.n * i.n * 8 for i in insts)
    host_in = [pinned_instance(torch, i) for i in insts] if e2e_reps > 0 else []
    host_out = pinned(torch, np.zeros(sum(i.n * i.n for i in insts))) if e2e_reps > 0 else None
    for r in range(e2e_reps + 1 if e2e_reps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with Batch.from_instances(host_in, stream=stream, tile_shape=tune["tile_shape"],
                                  schedule=tune.get("schedule", 0), tile_waves=tune["tile_waves"]) as BB:
            est, _ = BB.solve(tol_c=TOL_C, tol32=TOL32, tol64=TOL64)
            BB.get_values(out=host_out)
        torch.cuda.synchronize()
        if r > 0:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            e2e_nc += est["node_control_updates"]
    bounds = res / (1.0 - betas)
    umax = np.array([i.h_eff * i.cost / (1.0 - beta_of(i)) for i in insts])
    # error against the oracle at its stored sample of every instance (outside the
    # timed region; tests/golden/batched512.npz, written by the oracle-only script)
    gp = os.path.join(GOLDEN_DIR, "batched512.npz")
    g = np.load(gp) if os.path.exists(gp) else None

    def oracle_gate(vals):
        if g is None:
            return None
        off = np.concatenate([[0], np.cumsum(g["counts"])])
        errs = np.array([np.abs(vals[k][g["idx"][off[k]:off[k + 1]]] - g["u64"][off[k]:off[k + 1]]).max()
                         for k in range(len(insts))])
        gates = GATE_REL * np.maximum(1.0, np.array([np.abs(v).max() for v in vals]))
        return {"max_oracle_err": float(errs.max()), "max_err_over_gate": float((errs / gates).max()),
                "instances_within_gate": int((errs <= gates).sum()),
                "compared": f"{int(g['counts'][0])} seeded free nodes per instance (oracle FP64)"}

    vals = B.get_values()
    gate_oracle = oracle_gate(vals)
    certified = None
    if certify:
        # the solve to the one residual that certifies the gate of every instance,
        # min_i 0.99 gate_i (1 - beta_i), outside the timed region
        tol_cert = min(0.99 * GATE_REL * max(1.0, float(np.abs(v).max())) * (1.0 - beta_of(i))
                       for i, v in zip(insts, vals))
        e0, e1 = event_pair(torch, stream)
        e0.record(stream)
        cst, cres = B.solve(tol_c=TOL_C, tol32=TOL32, tol64=tol_cert, check_conv=False)
        e1.record(stream)
        torch.cuda.synchronize()
        certified = {"tol64_residual": tol_cert, "ms": e0.elapsed_time(e1), "status": cst["status"],
                     "fp64_passes": cst["fp64_passes"], "max_residual": float(cres.max()),
                     "oracle": oracle_gate(B.get_values())}
    plain_ms = []
    for _ in range(max(1, plain_reps)):
        flush_l2(flush)
        e0, e1 = event_pair(torch, stream)
        e0.record(stream)
        pst, pres = B.solve_full(tol32=TOL32, tol64=TOL64)
        e1.record(stream)
        torch.cuda.synchronize()
        plain_ms.append(e0.elapsed_time(e1))
    nodes32 = st["node_updates"] - st["fp64_node_updates"]
    # every instance has sigma > 0 (sigma ~ U[0, 0.1])
    parts = [(0.05, 32, nodes32)]
    B.close()
    patchy, plain = statistics.median(step_ms), statistics.median(plain_ms)
    return dict(
        value=value, step_ms=step_ms, launches=launches, clocks=clocks, insts=insts, n_free=n_free,
        tune=tune,
        summary={
            "time_to_1e-6_ms": {"patchy_batch": patchy, "plain_jacobi_fp32_batch": plain,
                                "speedup_vs_plain": plain / patchy},
            "value_gate": {"rule": "max |u - u_oracle| <= 1e-5 max(1, |u|) per instance at the oracle's "
                                   "stored sample; beside it the certified bound r / (1 - beta)",
                           "oracle": gate_oracle,
                           "certified_solve": certified,
                           "max_err_bound": float(bounds.max()),
                           "max_residual": float(res.max()),
                           "instances_within_bound": int((bounds <= GATE_REL * np.maximum(1.0, umax)).sum()),
                           "instances": len(insts)},
            "solver_stats": {"steps": st["fp32_passes"], "node_updates": st["node_updates"],
                             "fp64_node_updates": st["fp64_node_updates"],
                             "ms_fp32_passes": st["ms_stage"][0], "ms_residuals": st["ms_stage"][1],
                             "ms_fp64": st["ms_stage"][2], "ms_coarse": st["ms_stage"][3],
                             "ms_precompute": st["ms_stage"][4], "plain_sweeps": pst["sweeps"],
                             "plain_residual_max": float(pres.max())},
            "roofline": roofline_entry("k_wtiles<float> (FP32 patch passes, all instances)", parts,
                                       st["ms_stage"][0], peaks, WTILES_DRAM_BYTES.get("batched512")),
            "e2e": {"value": e2e_nc / (sum(e2e_ms) / 1e3) if e2e_ms else None, "unit": UNIT,
                    "ms_per_step": statistics.median(e2e_ms) if e2e_ms else None,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        })


# ------------------------------------------------------------ CPU baselines

def cpu_baseline(seconds: float, inst) -> dict:
    """The FP64 oracle as it stands (single-threaded Gauss-Seidel updates of the
    modified scheme) on a bounded sample of the workload: repeated Gauss-Seidel
    passes over the first rows of the grid (at most 2^20 nodes, from u = 0), as
    many as fit in about `seconds` seconds."""
    import oracle
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


def oracle_uhat(inst) -> np.ndarray:
    """u_hat of the instance from the oracle: the coarse solve (sigma = 0, from the
    big initial value) and its Q1 interpolation (Section 4.3, pre-computation),
    without the synthesis and the labels."""
    import oracle
    n, nc = inst.n, inst.coarse_n
    fine = oracle.Problem.from_instance(inst)
    sc, mc = oracle.coarse_data(n, nc, inst.speed, inst.mask)
    coarse = oracle.Problem(nc, inst.controls, sc, mc, h=inst.h_eff * (n - 1) / (nc - 1), lam=inst.lam,
                            sigma=0.0, cost=inst.cost, u_obstacle=fine.u_obstacle)
    uc, _, _ = coarse.solve(np.full(nc * nc, coarse.u_max), scheme=3, tol=1e-8)
    return oracle.interp_coarse(nc, uc, n, inst.mask, fine.u_obstacle)


def cpu_baseline_allcore(seconds: float, inst, plain_sweeps, golden=None) -> dict:
    """The all-core FP64 CPU baseline (oracle/cpu_parallel.c, OpenMP): full-grid
    Jacobi sweeps and u_hat-ordered Gauss-Seidel sweeps (one node list per block of
    rows) of eq. SLscheme3 on the whole grid, each for about seconds/2.  Time to
    solution is estimated from the time per sweep and a sweep count: for Jacobi
    the GPU comparator's (the same iteration from u = 0), for Gauss-Seidel the
    single-threaded oracle's count to its 1e-13 stop (stored with its solution)."""
    import oracle
    from oracle import cpu_parallel as cp
    A = cp.AllCore(inst)
    free = int((inst.mask == 0).sum())
    out = {"kind": "all-core FP64 Jacobi and u_hat-ordered Gauss-Seidel (OpenMP)",
           "cores": cp.threads(), "nproc": os.cpu_count(), "unit": UNIT}
    u = A.fix(np.zeros(A.N))
    v = np.empty_like(u)
    sweeps, t0 = 0, time.perf_counter()
    while sweeps == 0 or time.perf_counter() - t0 < seconds / 2:
        A.jacobi(u, v)
        u, v = v, u
        sweeps += 1
    dj = (time.perf_counter() - t0) / sweeps
    out["jacobi"] = {"ms_per_sweep": dj * 1e3, "value": free * inst.n_controls / dj, "sweeps_timed": sweeps}
    if plain_sweeps:
        out["jacobi"]["est_time_to_1e-6_s"] = dj * plain_sweeps
        out["jacobi"]["sweeps_for_estimate"] = int(plain_sweeps)
    uhat = oracle_uhat(inst)
    nodes, off = A.gs_lists(uhat)
    u = A.fix(uhat)
    sweeps, t0 = 0, time.perf_counter()
    while sweeps == 0 or time.perf_counter() - t0 < seconds / 2:
        A.gs(u, nodes, off)
        sweeps += 1
    dg = (time.perf_counter() - t0) / sweeps
    out["gs_uhat"] = {"ms_per_sweep": dg * 1e3, "value": free * inst.n_controls / dg, "sweeps_timed": sweeps,
                      "lists": int(off.size - 1)}
    if golden is not None:
        out["gs_uhat"]["est_time_to_1e-13_s"] = dg * int(golden["sweeps"])
        out["gs_uhat"]["sweeps_for_estimate"] = int(golden["sweeps"])
    out["value"] = max(out["jacobi"]["value"], out["gs_uhat"]["value"])
    out["sample"] = (f"{out['jacobi']['sweeps_timed']} Jacobi + {sweeps} Gauss-Seidel full-grid sweeps "
                     f"of {inst.name} on {out['cores']} threads")
    return out


# ------------------------------------------------------------ reference arm

def reference(args, ws, rank, local):
    """Reference arm: the FP64 oracle on the host cores, one bounded sample of the
    selected workload per step (Gauss-Seidel updates of a block of nodes)."""
    if rank != 0:
        return None
    import oracle
    if args.workload == "batched512":
        insts = [hi.batched_instance(1000 + k) for k in range(BATCH_COUNT)]
        n_free = sum(int((i.mask == 0).sum()) for i in insts)
        config = batched_config(insts, n_free, ws)
        # step k: one full sweep of instance k (about 0.1-0.7 s each)
        plan = [(insts[k % BATCH_COUNT], None) for k in range(args.warmup + args.steps)]
        what = "a full Gauss-Seidel sweep of one instance per step (instances 0, 1, ...)"
    else:
        insts = [inst for _, inst in make_instances(args.workload, args.n, args.coarse_n)]
        config = workload_config(args.workload, insts, ws)
        frac = 8 if args.workload == "patchy1025" else 64
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


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    d = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "source": "fallback"}
    if os.path.exists(p):
        d.update(json.load(open(p)))
        d["source"] = "measured"
    return d


def line(args, ws, value, step_ms, config) -> dict:
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(step_ms) / len(step_ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic", "config": config}


def ours(args, ws, rank, local):
    import torch

    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    stream = torch.cuda.current_stream()
    peaks = load_peaks()
    if args.workload == "batched512":
        B = bench_batched(steps=args.steps, warmup=args.warmup, plain_reps=args.plain_reps,
                          e2e_reps=args.e2e_reps, ws=ws, device=device, stream=stream, peaks=peaks,
                          certify=not args.no_certify)
        if rank != 0:
            return None
        out = line(args, ws, B["value"], B["step_ms"],
                   dict(batched_config(B["insts"], B["n_free"], ws), autotune=B["tune"]))
        out.update(B["summary"])
        out["gpu_launches"] = B["launches"]
        out["clocks"] = B["clocks"]
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.cpu_seconds, max(B["insts"], key=lambda i: i.n))
        return out

    labeled = make_instances(args.workload, args.n, args.coarse_n)
    labels = [lb for lb, _ in labeled]
    insts = [inst for _, inst in labeled]
    R = bench_single(args.workload, insts, labels, steps=args.steps, warmup=args.warmup,
                     plain_reps=args.plain_reps, e2e_reps=args.e2e_reps, certify=not args.no_certify,
                     ws=ws, device=device, stream=stream)
    out = line(args, ws, R["value"], R["step_ms"], workload_config(args.workload, insts, ws))
    out.update(single_summary(args.workload, insts, labels, R, peaks))
    out["gpu_launches"] = R["launches"]
    out["clocks"] = R["clocks"]
    if args.workload == "large4097" and not args.no_extras and not args.n:
        # the 1025^2 workload and the batch, with their own comparators, as extra keys
        ex = {}
        lab1 = make_instances("patchy1025")
        P1 = bench_single("patchy1025", [i for _, i in lab1], [lb for lb, _ in lab1],
                          steps=min(args.steps, 10), warmup=args.warmup, plain_reps=1, e2e_reps=3,
                          certify=not args.no_certify, ws=ws, device=device, stream=stream,
                          sample_clocks=False)
        ex["patchy1025"] = dict(config=workload_config("patchy1025", [i for _, i in lab1], ws),
                                value=P1["value"], ms_per_step=sum(P1["step_ms"]) / len(P1["step_ms"]),
                                steps=len(P1["step_ms"]), gpu_launches=P1["launches"],
                                **single_summary("patchy1025", [i for _, i in lab1],
                                                 [lb for lb, _ in lab1], P1, peaks))
        B = bench_batched(steps=min(args.steps, 5), warmup=3, plain_reps=1, e2e_reps=3, ws=ws,
                          device=device, stream=stream, peaks=peaks, sample_clocks=False,
                          certify=not args.no_certify)
        ex["batched512"] = dict(config=dict(batched_config(B["insts"], B["n_free"], ws), autotune=B["tune"]),
                                value=B["value"], ms_per_step=sum(B["step_ms"]) / len(B["step_ms"]),
                                steps=len(B["step_ms"]), gpu_launches=B["launches"], **B["summary"])
        out["extra"] = ex
    if rank != 0:
        return None
    if not args.no_cpu_baseline:
        main_inst = insts[1] if len(insts) > 1 else insts[0]
        lb = labels[1] if len(labels) > 1 else labels[0]
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds, main_inst)
        try:
            out["cpu_baseline_allcore"] = cpu_baseline_allcore(
                args.cpu_seconds, main_inst, R["plain"][lb]["sweeps"], load_golden(args.workload, main_inst))
        except (OSError, RuntimeError) as e:       # no C compiler / OpenMP on the host
            out["cpu_baseline_allcore"] = {"unavailable": str(e)[:200]}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--plain-reps", type=int, default=1)
    ap.add_argument("--e2e-reps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="large4097 only: skip the extra workloads")
    ap.add_argument("--no-certify", action="store_true", help="skip the solve to the certifying residual")
    ap.add_argument("--workload", choices=("large4097", "patchy1025", "batched512"), default="large4097",
                    help="large4097: the 4097^2 64-control workload with obstacles (default); "
                         "patchy1025: the 1025^2 three-sigma workload; batched512: 512 independent "
                         "instances of 65^2..513^2 solved as one batch")
    ap.add_argument("--n", type=int, default=0, help="fine grid size (profiling only)")
    ap.add_argument("--schedule", type=int, default=None,
                    help="hjb_desc.schedule for the patch solve (profiling only; default automatic)")
    ap.add_argument("--coarse-n", type=int, default=N_COARSE)
    args = ap.parse_args(argv)
    if args.schedule is not None:
        SOLVER_KW["schedule"] = args.schedule
    if args.warmup < 3 and args.impl == "ours":
        print("bench.py: --warmup must be >= 3", file=sys.stderr)
    ws, rank, local = dist_env()
    if args.impl == "reference":
        out = reference(args, ws, rank, local)
    else:
        out = ours(args, ws, rank, local)
    if out is not None:
        print(json.dumps(out), flush=True)
    if ws > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
