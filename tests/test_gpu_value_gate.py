"""Value gate of the benchmarked configurations against the FP64 oracle.

The benchmark times the patchy solve (and the plain Jacobi comparator) to an
FP64 sup-residual of 1e-6.  With beta = 1/(1 + lambda h) and h = dx the residual
alone bounds the error only by r / (1 - beta) (about 513 r at 1025^2, 2049 r at
4097^2), so these tests compare the results themselves with the oracle's
solution of the same instance (tests/golden/make_full_size.py: the FP64 oracle's
Gauss-Seidel value iteration of eq. SLscheme3 to a sup-increment of 1e-13):

* 1025^2, sigma in {0, 0.02, 0.1}: every node, at the FP32 gate
  1e-5 max(1, |u|), for the patchy solve and for the comparator, in the
  benchmark's own solver settings and tolerances;
* the same solve to a residual of 1e-13 (FP64 polish): the FP64 gate 1e-10 at
  the stored FP64 sample of nodes;
* the large recipe (64 controls, obstacles) at 2049^2: the seeded sample of
  65536 free nodes, for the benchmark's solve and for the solve to the residual
  that certifies the gate through r / (1 - beta); at 4097^2 the certified bound;
* the 512-instance batch at its 256 sampled nodes per instance.
"""
import os
import sys

import numpy as np
import pytest

import hjb_inputs as hi

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def _golden(name):
    p = os.path.join(GOLDEN, name + ".npz")
    if not os.path.exists(p):
        pytest.fail(f"missing oracle solution {p}: run tests/golden/make_full_size.py")
    return dict(np.load(p))


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the -m gpu tests")
    from paper_1502_01629_gb300 import build
    build.build()
    return torch


def _gate(u):
    return 1e-5 * max(1.0, float(np.abs(u).max()))


@pytest.mark.parametrize("sigma", [0.0, 0.02, 0.1])
def test_patchy_1025_full_size_meets_the_fp32_gate(sigma):
    _gpu()
    from paper_1502_01629_gb300 import Problem
    B = _bench()
    inst = hi.patchy_1025(sigma)
    g = _golden(f"patchy1025_sigma{sigma:g}")
    assert int(g["n"]) == inst.n
    ref = g["u32"].astype(np.float64)
    with Problem.from_instance(inst, **B.SOLVER_KW) as P:
        P.coarse_solve(tol_c=B.TOL_C)
        P.build_patches()
        st = P.solve_patches(tol32=B.TOL32, tol64=B.TOL64)
        assert st["residual"] <= B.TOL64
        u = P.get_value()
        err = np.abs(u - ref)
        assert err.max() <= _gate(u), (sigma, float(err.max()), int(err.argmax()))
        # the comparator in the benchmark's settings meets the same gate
        sf = P.solve_full(precision=32, tol=B.TOL32, tol64=B.TOL64)
        assert sf["residual"] <= B.TOL64
        v = P.get_value()
        errv = np.abs(v - ref)
        assert errv.max() <= _gate(v), (sigma, float(errv.max()))
        # the oracle's error report of the benchmark agrees with this comparison
        rep = B.value_gate(u, inst, st["residual"], g)
        assert rep["pass"] and abs(rep["oracle_err"] - float(err.max())) == 0.0


@pytest.mark.parametrize("sigma", [0.0, 0.1])
def test_patchy_1025_fp64_polish_meets_the_fp64_gate(sigma):
    _gpu()
    from paper_1502_01629_gb300 import Problem
    B = _bench()
    inst = hi.patchy_1025(sigma)
    g = _golden(f"patchy1025_sigma{sigma:g}")
    with Problem.from_instance(inst, **B.SOLVER_KW) as P:
        P.coarse_solve(tol_c=B.TOL_C)
        P.build_patches()
        st = P.solve_patches(tol32=B.TOL32, tol64=1e-13)
        assert st["residual"] <= 1e-13
        u = P.get_value()
    err = np.abs(u[g["idx"]] - g["u64"]).max()
    assert err <= 1e-10, (sigma, float(err))


def test_large_2049_sampled_nodes_against_the_oracle():
    """The large recipe (64 controls, obstacles, sigma = 0.01) at 2049^2, solved
    with the 4097^2 benchmark's settings, at the oracle's 65536 seeded free
    nodes (tests/golden/large2049_sigma0.01.npz: FP64 Gauss-Seidel on every
    core by nested grids, certified by the scalar oracle's residual).  The
    solve to the benchmark's residual 1e-6 is bounded only by r / (1 - beta)
    (1025 r here); its error is reported against the gate, and the solve to the
    certifying residual meets the gate at every sampled node."""
    _gpu()
    from paper_1502_01629_gb300 import Problem
    B = _bench()
    inst = hi.large_instance(n=2049)
    g = _golden("large2049_sigma0.01")
    assert int(g["n"]) == inst.n
    # the stored solution's own certificate is far inside the gate
    assert float(g["residual"]) / (1.0 - B.beta_of(inst)) <= 1e-8
    idx = g["idx"]
    with Problem.from_instance(inst, **B.SOLVER_KW) as P:
        P.coarse_solve(tol_c=B.TOL_C)
        P.build_patches()
        st = P.solve_patches(tol32=B.TOL32, tol64=B.TOL64)
        assert st["residual"] <= B.TOL64
        u = P.get_value()
        err = np.abs(u[idx] - g["u64"]).max()
        assert err <= 2.0 * _gate(u), float(err)
        tol = B.certify_tol(inst)
        P.coarse_solve(tol_c=B.TOL_C)
        P.build_patches()
        st2 = P.solve_patches(tol32=B.TOL32, tol64=tol)
        assert st2["residual"] <= tol
        w = P.get_value()
        err2 = np.abs(w[idx] - g["u64"]).max()
        assert err2 <= st2["residual"] / (1.0 - B.beta_of(inst)) + 1e-9 and err2 <= _gate(w), float(err2)


def test_large_4097_certified_solve_meets_the_bound():
    """At 4097^2 no stored oracle solution exists (the oracle's Gauss-Seidel on
    this grid takes thousands of sweeps); the benchmark's solve reaches the FP64
    residual 1e-6 and the solve to the certifying residual r bounds the error by
    r / (1 - beta) <= the FP32 gate (the FP64 residual kernel is the one checked
    against the oracle's operator at every node of the smaller grids)."""
    _gpu()
    from paper_1502_01629_gb300 import Problem
    B = _bench()
    inst = hi.large_instance()
    with Problem.from_instance(inst, **B.SOLVER_KW) as P:
        P.coarse_solve(tol_c=B.TOL_C)
        P.build_patches()
        st = P.solve_patches(tol32=B.TOL32, tol64=B.TOL64)
        assert st["residual"] <= B.TOL64
        u = P.get_value()
        tol = B.certify_tol(inst)
        P.coarse_solve(tol_c=B.TOL_C)
        P.build_patches()
        st2 = P.solve_patches(tol32=B.TOL32, tol64=tol)
        assert st2["residual"] <= tol
        w = P.get_value()
        bound = st2["residual"] / (1.0 - B.beta_of(inst))
        assert bound <= _gate(w)
        # the two solves agree within the first one's own bound
        assert np.abs(u - w).max() <= st["residual"] / (1.0 - B.beta_of(inst)) + bound


def test_large_4097_sigma0_worklist_ends_and_the_fp64_stage_decides():
    """sigma = 0 on the large recipe: FP32 rounding keeps a few tiles changing by
    more than tol32 (6.6e-7 against 1.25e-7), so the worklist stops putting them
    back after their visit cap; the solve must end in bounded time, report the
    FP32 phase as not converged without an FP64 stage, and with one reach the
    FP64 residual (which then decides the status)."""
    _gpu()
    import time
    from paper_1502_01629_gb300 import HJB_ERR_NOT_CONVERGED, Problem
    B = _bench()
    inst = hi.large_instance(sigma=0.0)
    with Problem.from_instance(inst, **B.SOLVER_KW) as P:
        P.coarse_solve(tol_c=B.TOL_C)
        P.build_patches()
        t0 = time.time()
        st = P.solve_patches(tol32=B.TOL32, tol64=B.TOL64)
        assert time.time() - t0 < 10.0
        assert st["status"] == 0 and 0.0 <= st["residual"] <= B.TOL64
        u = P.get_value()
        assert np.isfinite(u).all()
        P.coarse_solve(tol_c=B.TOL_C)
        P.build_patches()
        t0 = time.time()
        s0 = P.solve_patches(tol32=B.TOL32, tol64=0.0, check_conv=False)
        assert time.time() - t0 < 10.0
        assert s0["status"] in (0, HJB_ERR_NOT_CONVERGED)
        # the values after the capped FP32 phase are within the FP32 gate of the
        # converged ones
        v = P.get_value()
        assert np.abs(v - u).max() <= _gate(u)


@pytest.mark.parametrize("schedule", [0, 3])
def test_batched_512_sampled_nodes_against_the_oracle(schedule):
    """The 512-instance workload in one batch (barrier tiles and the worklist, the
    autotuner's two families), every instance at the oracle's 256 seeded free
    nodes (tests/golden/batched512.npz, the FP64 oracle to a sup-increment of
    1e-13).  At the benchmark's FP64 residual 1e-6 the error is bounded only by
    r / (1 - beta) (up to 5e-4 for lambda = 0.5 at 513^2): nearly every instance
    meets the FP32 gate and the rest stay within twice it.  Solved to the
    residual that certifies the gate for every instance (min_i of
    0.99 gate_i (1 - beta_i), gate_i from the first solve's values), every
    instance meets it."""
    _gpu()
    from paper_1502_01629_gb300 import Batch
    B = _bench()
    g = _golden("batched512")
    insts = [hi.batched_instance(1000 + k) for k in range(len(g["counts"]))]
    off = np.concatenate([[0], np.cumsum(g["counts"])])

    def ratios(vals):
        return np.array([np.abs(v[g["idx"][off[k]:off[k + 1]]] - g["u64"][off[k]:off[k + 1]]).max() / _gate(v)
                         for k, v in enumerate(vals)])

    with Batch.from_instances(insts, schedule=schedule) as bt:
        st, res = bt.solve(tol_c=B.TOL_C, tol32=B.TOL32, tol64=B.TOL64)
        assert st["status"] == 0 and (res <= B.TOL64).all()
        vals = bt.get_values()
        r = ratios(vals)
        assert (r <= 1.0).mean() >= 0.97 and r.max() <= 2.0, (int((r > 1).sum()), float(r.max()))
        tol = min(0.99 * _gate(v) * (1.0 - B.beta_of(i)) for i, v in zip(insts, vals))
        st, res = bt.solve(tol_c=B.TOL_C, tol32=B.TOL32, tol64=tol)
        assert st["status"] == 0 and (res <= tol).all()
        r = ratios(bt.get_values())
        assert r.max() <= 1.0, (int((r > 1).sum()), float(r.max()))
