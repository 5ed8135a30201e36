"""The all-core FP64 CPU baseline (oracle/cpu_parallel.c) solves the same scheme:
its Jacobi sweeps from 0 and its u_hat-ordered Gauss-Seidel sweeps (one list per
block of rows, threads in parallel) reach the oracle's fixed point of eq.
SLscheme3, with obstacles and with a drift, and one Jacobi sweep is the oracle's
operator application."""
import numpy as np
import pytest

import hjb_inputs as hi
import oracle
from oracle import cpu_parallel as cp


def _cases():
    d = hi.disc_instance(41, 0.05, n_controls=16, speed=hi.speed_sine(41), lam=0.8, coarse_n=11)
    rng = np.random.default_rng(3)
    d.drift = rng.uniform(-0.3, 0.3, 2 * 41 * 41).astype(np.float32)
    return {"patchy-s0.02": hi.patchy_1025(0.02, n=65, coarse_n=17),
            "obstacles": hi.large_instance(n=65, coarse_n=17),
            "drift": d}


@pytest.mark.parametrize("case", ["patchy-s0.02", "obstacles", "drift"])
def test_allcore_sweeps_reach_the_oracle_fixed_point(case):
    inst = _cases()[case]
    O = oracle.Problem.from_instance(inst)
    ref, _, _ = O.solve(scheme=3, tol=1e-14)
    A = cp.AllCore(inst)
    u = A.fix(np.zeros(A.N))
    # one Jacobi sweep is one application of the oracle's operator
    v = np.empty_like(u)
    A.jacobi(u, v)
    Tu, _, _ = O.apply(O.fix_nonfree(np.zeros(O.N)), scheme=3)
    np.testing.assert_allclose(v, Tu, rtol=0, atol=1e-13)
    for _ in range(20000):
        inc = A.jacobi(u, v)
        u, v = v, u
        if inc < 1e-14:
            break
    assert np.abs(u - ref).max() < 1e-11
    pre = oracle.patchy_precompute(inst, tol_c=1e-10)
    nodes, off = A.gs_lists(pre["uhat"], lists=4)
    assert np.array_equal(np.sort(nodes), np.flatnonzero(inst.mask == 0))
    w = A.fix(pre["uhat"])
    for _ in range(20000):
        if A.gs(w, nodes, off) < 1e-14:
            break
    assert np.abs(w - ref).max() < 1e-11
