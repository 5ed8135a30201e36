"""Host arithmetic of bench.py (CPU): the roofline fractions recompute from the
line's own fields, the value gate compares against the stored oracle solutions
the way its report says, the certifying residual's bound meets the gate, and a
stored solution is only used for the instance (size and sigma) it belongs to."""
import os
import sys
from types import SimpleNamespace

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import hjb_inputs as hi  # noqa: E402


def test_roofline_fractions_recompute_from_the_counts():
    peaks = {"sm_max_mhz": 2000.0, "source": "measured"}
    parts = [(0.1, 32, 1_000_000), (0.0, 32, 2_000_000)]
    ms = 4.0
    r = bench.roofline_entry("k", parts, ms, peaks, traffic=123.0)
    t = ms / 1e3
    ops = 1_000_000 * 32 * 60 + 2_000_000 * 32 * 18
    words = 1_000_000 * 32 * 16 + 2_000_000 * 32 * 4
    fp32_peak = 152 * 128 * 2 * 2000e6 / 1e12
    smem_peak = 152 * 32 * 2000e6 / 1e12
    assert r["frac_fp32"] == pytest.approx(ops / t / 1e12 / fp32_peak, rel=1e-12)
    assert r["frac_lsu"] == pytest.approx(words / t / 1e12 / smem_peak, rel=1e-12)
    assert r["frac"] == max(r["frac_fp32"], r["frac_lsu"])
    assert r["achieved"] / r["peak"] == pytest.approx(r["frac"], rel=1e-12)
    assert r["fp32_node_control_updates"] == 3_000_000 * 32 and r["traffic"] == 123.0


def _inst(n=33, lam=1.0, sigma=0.0, cost=1.0):
    return SimpleNamespace(n=n, lam=lam, sigma=sigma, cost=cost, h_eff=2.0 / (n - 1))


def test_value_gate_against_every_node_and_against_samples():
    inst = _inst()
    u = np.linspace(0.0, 0.9, inst.n * inst.n)
    ref = u.astype(np.float32)
    err = np.zeros_like(u)
    err[17] = 3e-6
    g_all = {"u32": ref, "residual": np.float64(1e-15)}
    rep = bench.value_gate(u + err, inst, 1e-9, g_all)
    assert rep["oracle_err"] == pytest.approx(np.abs(u + err - ref.astype(np.float64)).max())
    assert rep["pass"] and rep["gate"] == 1e-5
    assert rep["err_bound"] == pytest.approx(1e-9 / (1.0 - bench.beta_of(inst)))
    # a sampled solution that misses the erroneous node does not see it; one that
    # holds it does, and a large error fails the gate
    idx = np.array([3, 17, 40])
    g_s = {"idx": idx, "u64": u[idx], "residual": np.float64(1e-15)}
    big = np.zeros_like(u)
    big[40] = 2e-5
    rep2 = bench.value_gate(u + big, inst, 1e-9, g_s)
    assert rep2["oracle_err"] == pytest.approx(2e-5) and not rep2["pass"]
    assert rep2["compared"].startswith("3 seeded")
    # without a stored solution the certified bound decides
    rep3 = bench.value_gate(u, inst, 1e-9, None)
    assert rep3["pass"] == (rep3["err_bound"] <= rep3["gate"])


@pytest.mark.parametrize("make", [lambda: hi.patchy_1025(0.1, n=129, coarse_n=17),
                                  lambda: hi.large_instance(n=129, coarse_n=33)])
def test_certifying_residual_bound_meets_the_gate(make):
    inst = make()
    tol = bench.certify_tol(inst)
    # |u| <= h l / (1 - beta); the bound r / (1 - beta) at r = tol is within the gate
    # of that bound, and the gate of any value field is at least 1e-5
    umax = inst.h_eff * inst.cost / (1.0 - bench.beta_of(inst))
    assert tol / (1.0 - bench.beta_of(inst)) <= bench.GATE_REL * max(1.0, umax)
    assert tol > 0


def test_stored_solutions_belong_to_their_instance():
    n1025 = SimpleNamespace(n=1025, sigma=0.02)
    g = bench.load_golden("patchy1025", n1025)
    assert g is not None and int(g["n"]) == 1025 and g["u32"].size == 1025 * 1025
    assert bench.load_golden("patchy1025", SimpleNamespace(n=129, sigma=0.02)) is None
    assert bench.golden_name("large4097", SimpleNamespace(n=2049, sigma=0.01)) == "large2049_sigma0.01"
    g2 = bench.load_golden("large4097", SimpleNamespace(n=2049, sigma=0.01))
    assert g2 is not None and g2["idx"].size == g2["u64"].size == 65536
    assert bench.load_golden("large4097", SimpleNamespace(n=4097, sigma=0.01)) is None
