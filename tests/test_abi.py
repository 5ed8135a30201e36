"""The C-ABI library builds for sm_103a, loads, exports every entry point the
header declares, and rejects bad input on the host without touching a GPU.
The regime helper (Section 4.1) is checked against the paper's printed values."""
import ctypes
import json
import math
import os

import numpy as np
import pytest

import hjb_inputs as hi
from paper_1502_01629_gb300 import build as gbuild

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


@pytest.fixture(scope="module")
def L():
    gbuild.build()
    from paper_1502_01629_gb300 import _lib
    return _lib


def test_every_declared_symbol_is_exported_and_bound(L):
    names = L.header_functions()
    assert len(names) >= 20
    lib = L.lib()
    for name in names:
        assert hasattr(lib, name), name
        assert name in L._SIGNATURES, f"{name} has no binding"


def test_status_strings(L):
    lib = L.lib()
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert lib.hjb_status_string(code)
    assert lib.hjb_status_string(-99) == b"unknown status"
    lib.hjb_destroy(None)


def _create(L, desc, speed, mask, controls, sector=None, drift=None):
    h = ctypes.c_void_p()
    p = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
    return L.lib().hjb_create_problem(ctypes.byref(desc), p(speed), p(mask), p(sector),
                                      p(controls), p(drift), None, ctypes.byref(h))


def _desc(L, **kw):
    d = L.Desc()
    d.n, d.n_controls, d.h, d.lam, d.sigma, d.cost = 9, 4, 0.0, 1.0, 0.0, 1.0
    d.coarse_n, d.n_patches, d.scheme, d.band_width, d.band_window = 0, 1, 3, 1.0, 8
    d.band_group, d.wave_warps, d.resort_passes = 1, 0, 0
    d.schedule, d.tile_waves, d.tile_period, d.local_sweeps = 0, 8, 8, 1
    d.tile_shape = 0
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("bad", [
    dict(n=2), dict(n_controls=0), dict(n_controls=300), dict(lam=-1.0), dict(sigma=-0.1),
    dict(cost=0.0), dict(scheme=4), dict(n_patches=0), dict(coarse_n=4),
    dict(lam=float("nan")), dict(visit=5), dict(visit=-1), dict(resort_passes=-1), dict(schedule=5), dict(tile_shape=3), dict(tile_shape=-2),
])
def test_invalid_descriptions_are_rejected_on_host(L, bad):
    d = _desc(L, **bad)
    n = max(d.n, 3)
    rc = _create(L, d, np.ones(n * n, np.float32), np.zeros(n * n, np.uint8), hi.control_set(4))
    assert rc == L.HJB_ERR_INVALID_ARG
    assert L.lib().hjb_last_error()


def test_invalid_host_arguments_are_rejected(L):
    """Arguments checked on the host before any device work: missing arrays and
    a non-finite control.  (The per-node arrays are checked on the device after
    the upload; tests/test_gpu_parity.py covers those.)"""
    n = 9
    d = _desc(L)
    ctr = hi.control_set(4)
    sp = np.ones(n * n, np.float32)
    mk = np.zeros(n * n, np.uint8)
    bad_ctr = ctr.copy(); bad_ctr[1, 0] = np.inf
    assert _create(L, d, sp, mk, bad_ctr) == L.HJB_ERR_INVALID_ARG
    assert _create(L, d, None, mk, ctr) == L.HJB_ERR_INVALID_ARG
    assert _create(L, d, sp, None, ctr) == L.HJB_ERR_INVALID_ARG


def test_regime_matches_paper_thresholds(L):
    """Section 5.4: eikonal eps < dx/4 (Upsilon = 1) and Zermelo eps < dx/120
    (f_min = 1/6, f_max = 3/2, Upsilon = 9), with the printed tau values."""
    from paper_1502_01629_gb300 import regime
    g = json.load(open(GOLDEN))
    for case in ("eikonal_thresholds", "zermelo_thresholds"):
        c = g[case]
        for dx, tau in zip(c["dx"], c["tau"]):
            r = regime(dx, c["f_min"], c["f_max"], 0.0)
            assert math.isclose(r["upsilon"], c["upsilon"], rel_tol=1e-12)
            # the condition 1/omega < dx/(1+Upsilon) with omega = f_min/(2 eps)
            # reads eps < f_min dx / (2 (1 + Upsilon))
            assert math.isclose(r["eps_threshold"], tau, rel_tol=1e-9)
            assert math.isclose(r["eps_threshold"] / dx, c["eps_over_dx_bound"], rel_tol=1e-9)
            below = regime(dx, c["f_min"], c["f_max"], 0.9 * tau)
            above = regime(dx, c["f_min"], c["f_max"], 1.1 * tau)
            assert below["holds"] == 1 and above["holds"] == 0


def test_regime_alpha_choice_is_inside_the_bounds(L):
    """Section 4.1: alpha = 1/(1+Upsilon) lies in (alpha_lower, alpha_upper) whenever the
    condition holds, and then h = alpha dx / f_min meets both eq. upper-bound and
    eq. lower-bound."""
    from paper_1502_01629_gb300 import regime
    rng = np.random.default_rng(0)
    for _ in range(200):
        dx = 10 ** rng.uniform(-3, -1)
        fmin = rng.uniform(0.1, 2.0)
        fmax = fmin * rng.uniform(1.0, 10.0)
        eps = 10 ** rng.uniform(-9, -2)
        r = regime(dx, fmin, fmax, eps)
        if r["holds"]:
            assert r["alpha_lower"] < r["alpha"] < r["alpha_upper"] < 1.0 / r["upsilon"]
            assert r["upper_ok"] == 1 and r["lower_ok"] == 1
        else:
            assert not (r["upper_ok"] and r["lower_ok"])
