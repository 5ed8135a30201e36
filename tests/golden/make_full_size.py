#!/usr/bin/env python3
"""Write the full-size oracle solutions the value-gate tests compare against.

Calls only ``oracle/`` (the FP64 CPU oracle) and the seeded input generators of
``hjb_inputs``; nothing here touches the CUDA solver.

    python tests/golden/make_full_size.py patchy1025    # three files, one per sigma
    python tests/golden/make_full_size.py large4097     # sampled nodes only
    python tests/golden/make_full_size.py large4097 --allcore   # the same on every core
    python tests/golden/make_full_size.py large2049     # the large recipe at 2049^2, every core
    python tests/golden/make_full_size.py batched512    # 256 sampled nodes per instance

What is solved: the fixed point u* of eq. SLscheme3 (Section 3; the same fixed
point as eq. SLscheme2 by the Section 3 proof) on the workload's grid, by the
oracle's Gauss-Seidel value iteration in increasing u_hat (Section 4.3: the
nodes ordered by the interpolated coarse solution; the order changes the speed
only), started from u_hat and stopped at a sup-increment <= 1e-13.  For
Gauss-Seidel of a beta-contraction the error after a sweep whose increment is
d is at most d beta / (1 - beta): 5e-11 at 1025^2, 2e-10 at 4097^2.

``--allcore`` (4097^2): the same iteration on every host core
(oracle/cpu_parallel.c: one node list per block of rows, each in increasing
order of the start value, the lists relaxed concurrently in place, a chaotic
relaxation of the same contraction), by nested grids: the same recipe at 257^2
from the oracle's u_hat, then 1025^2, 2049^2 and 4097^2, each started from (and
ordered by) the bilinear interpolation of the previous level's solution (the start and
order change the speed only; from the 129^2 coarse u_hat the 4097^2
Gauss-Seidel has a slow phase of hundreds of sweeps).  Then the single-threaded
oracle's residual r = ||T2 u - u|| of the result, which bounds the error by
r / (1 - beta) whatever the order of the updates was; the file records r.

Stored per workload and sigma (``tests/golden/<name>.npz``):
  u32        -- u* rounded to float32, every node (1025^2 only): enough for the
                FP32 gate 1e-5 max(1, |u|) (rounding 6e-8 |u|);
  idx, u64   -- a seeded sample of free nodes and u* there in float64, for the
                1e-10 gate after the FP64 polish;
  sum64      -- sum of u* over all nodes in float64 (a checksum of the file);
  sweeps, last_increment, residual -- the oracle's own convergence record
                (residual = ||T2 u - u|| over the free nodes, eq. SLscheme2).
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

TOL = 1e-13
SIGMAS_1025 = (0.0, 0.02, 0.1)
N_SAMPLES = {"patchy1025": 8192, "large4097": 65536, "batched512": 256}
BATCH_COUNT = 512


def golden_path(name: str) -> str:
    return os.path.join(HERE, name + ".npz")


def patchy1025_name(sigma: float) -> str:
    return f"patchy1025_sigma{sigma:g}"


def large4097_name() -> str:
    return "large4097_sigma0.01"


def large_name(n: int) -> str:
    return f"large{n}_sigma0.01"


def sample_nodes(mask: np.ndarray, count: int, seed: int = 20260) -> np.ndarray:
    """A seeded sorted sample of free nodes (mask 0)."""
    free = np.flatnonzero(mask == 0)
    rng = np.random.default_rng(np.random.PCG64(seed))
    return np.sort(rng.choice(free, size=min(count, free.size), replace=False)).astype(np.int64)


def solve_one(job):
    workload, sigma = job
    import hjb_inputs as hi
    import oracle
    if workload == "patchy1025":
        inst = hi.patchy_1025(sigma)
        name = patchy1025_name(sigma)
    else:
        inst = hi.large_instance()
        name = large4097_name()
    t0 = time.time()
    pre = oracle.patchy_precompute(inst, tol_c=1e-10)
    O = pre["fine"]
    order = np.argsort(pre["uhat"], kind="stable")
    u, sweeps, last = O.solve(u0=O.fix_nonfree(pre["uhat"]), scheme=3, method="gs",
                              order=order, tol=TOL, max_sweeps=200000)
    if sweeps < 0:
        raise RuntimeError(f"{name}: the oracle did not reach {TOL}")
    res = O.residual(u)
    idx = sample_nodes(inst.mask, N_SAMPLES[workload])
    out = dict(idx=idx, u64=u[idx], sum64=np.float64(u.sum()), sweeps=np.int64(sweeps),
               last_increment=np.float64(last), residual=np.float64(res),
               n=np.int64(inst.n), sigma=np.float64(inst.sigma))
    if workload == "patchy1025":
        out["u32"] = u.astype(np.float32)
    np.savez_compressed(golden_path(name), **out)
    return f"{name}: {sweeps} sweeps, last increment {last:.2e}, residual {res:.2e}, {time.time() - t0:.0f} s"


def _allcore_gs(inst, u0, key, tol, name, t0):
    from oracle import cpu_parallel as cp
    A = cp.AllCore(inst)
    u = A.fix(u0)
    nodes, off = A.gs_lists(key)
    sweeps, last = 0, np.inf
    while last > tol and sweeps < 200000:
        last = A.gs(u, nodes, off)
        sweeps += 1
        if sweeps % 25 == 0:
            print(f"  {name} n={inst.n}: sweep {sweeps}, increment {last:.3e}, {time.time() - t0:.0f} s",
                  flush=True)
    if last > tol:
        raise RuntimeError(f"{name}: no convergence to {tol} at n={inst.n}")
    return u, sweeps, last


def solve_large_allcore(levels=(257, 1025, 4097)):
    """The large recipe at levels[-1]^2 on every core by nested grids; the
    stored residual is the scalar oracle's."""
    import hjb_inputs as hi
    import oracle
    from oracle import cpu_parallel as cp
    name = large_name(levels[-1])
    t0 = time.time()
    u, prev = None, None
    for n in levels:
        inst = hi.large_instance(n=n, coarse_n=(n - 1) // 32 + 1 if n > 257 else (n - 1) // 8 + 1)
        O = oracle.Problem.from_instance(inst)
        if prev is None:
            start = oracle.patchy_precompute(inst, tol_c=1e-10)["uhat"]
        else:
            start = oracle.interp_coarse(prev.n, u, n, inst.mask, O.u_obstacle)
        tol = TOL if n == levels[-1] else 1e-10
        u, sweeps, last = _allcore_gs(inst, O.fix_nonfree(start), start, tol, name, t0)
        print(f"  {name}: level n={n} done, {sweeps} sweeps, {time.time() - t0:.0f} s", flush=True)
        prev = inst
    res = O.residual(u)
    idx = sample_nodes(inst.mask, N_SAMPLES["large4097"])
    np.savez_compressed(golden_path(name), idx=idx, u64=u[idx], sum64=np.float64(u.sum()),
                        sweeps=np.int64(sweeps), last_increment=np.float64(last),
                        residual=np.float64(res), n=np.int64(inst.n), sigma=np.float64(inst.sigma),
                        allcore=np.int64(cp.threads()), levels=np.array(levels, np.int64),
                        coarse_n=np.int64(inst.coarse_n))
    print(f"{name}: {sweeps} all-core sweeps at n={inst.n} on {cp.threads()} threads, last increment "
          f"{last:.2e}, oracle residual {res:.2e}, {time.time() - t0:.0f} s", flush=True)


def solve_batch_instance(k):
    """Instance k of the 512-instance workload (seed 1000 + k): the oracle's
    solution at a seeded sample of its free nodes."""
    import hjb_inputs as hi
    import oracle
    inst = hi.batched_instance(1000 + k)
    pre = oracle.patchy_precompute(inst, tol_c=1e-10)
    O = pre["fine"]
    order = np.argsort(pre["uhat"], kind="stable")
    u, sweeps, last = O.solve(u0=O.fix_nonfree(pre["uhat"]), scheme=3, method="gs",
                              order=order, tol=TOL, max_sweeps=200000)
    if sweeps < 0:
        raise RuntimeError(f"batched instance {k}: the oracle did not reach {TOL}")
    idx = sample_nodes(inst.mask, N_SAMPLES["batched512"], seed=20260 + k)
    return k, idx, u[idx], sweeps, O.residual(u)


def main_batched(workers: int):
    t0 = time.time()
    res = [None] * BATCH_COUNT
    with mp.get_context("spawn").Pool(workers) as pool:
        for k, idx, vals, sweeps, r in pool.imap_unordered(solve_batch_instance, range(BATCH_COUNT)):
            res[k] = (idx, vals, sweeps, r)
    counts = np.array([r[0].size for r in res], np.int64)
    np.savez_compressed(golden_path("batched512"),
                        counts=counts, idx=np.concatenate([r[0] for r in res]),
                        u64=np.concatenate([r[1] for r in res]),
                        sweeps=np.array([r[2] for r in res], np.int64),
                        residual=np.array([r[3] for r in res]))
    print(f"batched512: {BATCH_COUNT} instances, max residual {max(r[3] for r in res):.2e}, "
          f"{time.time() - t0:.0f} s", flush=True)


def main(argv):
    which = argv[1] if len(argv) > 1 else "patchy1025"
    if which == "patchy1025":
        jobs = [("patchy1025", s) for s in SIGMAS_1025]
    elif which == "large4097" and "--allcore" in argv:
        return solve_large_allcore((257, 1025, 2049, 4097))
    elif which == "large2049":
        return solve_large_allcore((257, 1025, 2049))
    elif which == "large4097":
        jobs = [("large4097", 0.01)]
    elif which == "batched512":
        return main_batched(int(argv[2]) if len(argv) > 2 else max(1, (os.cpu_count() or 2) - 1))
    else:
        raise SystemExit("usage: make_full_size.py patchy1025|large4097 [--allcore]|large2049|batched512 [workers]")
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        for line in pool.imap_unordered(solve_one, jobs):
            print(line, flush=True)


if __name__ == "__main__":
    main(sys.argv)
