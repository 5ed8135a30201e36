"""The seeded input generators: shapes, dtypes, determinism and the closed-form
fields of the paper's problems (Section 5), checked against their definitions
on the CPU."""
import math

import numpy as np
import pytest

import hjb_inputs as hi


def test_instances_are_deterministic_and_well_formed():
    for make in (lambda: hi.batched_instance(1007), lambda: hi.warmstart_instance(100003, n=129, coarse_n=65),
                 lambda: hi.large_instance(n=257, coarse_n=65)):
        a, b = make(), make()
        n = a.n
        assert a.speed.dtype == np.float32 and a.speed.shape == (n * n,)
        assert a.mask.dtype == np.uint8 and a.sector.dtype == np.int8
        np.testing.assert_array_equal(a.speed, b.speed)
        np.testing.assert_array_equal(a.mask, b.mask)
        np.testing.assert_array_equal(a.sector, b.sector)
        assert set(np.unique(a.mask)) <= {0, 1, 2}
        tgt = a.mask == hi.MASK_TARGET
        assert (a.sector[tgt] >= 0).all() and (a.sector[tgt] < a.n_patches).all()
        assert (a.sector[~tgt] == -1).all()
        if a.coarse_n:
            assert (a.n - 1) % (a.coarse_n - 1) == 0


def test_batched_sizes_nest_with_ratio_four():
    for seed in range(1000, 1040):
        x = hi.batched_instance(seed)
        assert 65 <= x.n <= 513 and (x.n - 1) % 8 == 0
        assert (x.n - 1) % (x.coarse_n - 1) == 0


@pytest.mark.parametrize("n,fmax,eps", [(51, 2.0, 0.1), (101, 1.5, 1e-3), (201, 1.0, 1e-2)])
def test_time_step_meets_the_upper_bound(n, fmax, eps):
    """h f_max + sqrt(2 eps h) = 0.9 dx (Section 4.1, eq. upper-bound with a margin)."""
    h = hi.h_upper_bound(n, fmax, eps)
    dx = 2.0 / (n - 1)
    assert abs(h * fmax + math.sqrt(2.0 * eps * h) - 0.9 * dx) <= 1e-12


def test_general_problem_fields_follow_their_definitions():
    """eq. nonomog, eq. s123 and eq. l123 at every node, from the coordinates."""
    n = 41
    X1, X2 = hi.mesh(n)
    X1, X2 = X1.reshape(-1), X2.reshape(-1)
    x3 = hi.general_instance(n, 3, 3, eps=0.1)
    np.testing.assert_array_equal(x3.speed, (1.0 + np.maximum(X2, np.maximum(X1, 0.0))).astype(np.float32))
    up = X2 >= 0.0
    np.testing.assert_array_equal(x3.sigma_field, np.where(up, math.sqrt(0.1), 0.0).astype(np.float32))
    assert x3.diffusion == 1 and hi.general_instance(n, 2, 1).diffusion == 0
    np.testing.assert_array_equal(x3.cost_field, (1.0 + np.abs(X1 * X2)).astype(np.float32))
    a = x3.controls
    np.testing.assert_allclose(x3.control_cost, np.abs(a[:, 0] / (2.0 + a[:, 1])), rtol=0, atol=0)
    x1 = hi.general_instance(n, 1, 1)
    assert x1.sigma_field is None and x1.cost_field is None and x1.control_cost is None
    # boundary target, the four sides as sectors, no discount
    m = x1.mask.reshape(n, n)
    assert (m[0] == 1).all() and (m[-1] == 1).all() and (m[:, 0] == 1).all() and (m[:, -1] == 1).all()
    assert (m[1:-1, 1:-1] == 0).all() and x1.lam == 0.0 and x1.n_patches == 4


def test_zermelo_speeds_span_the_paper_range():
    """|f| = |R_theta x/|x| + (eta/2) a| / (1 + |x|^2): at most 3/2 (near the origin
    with a aligned) and at least 1/6 (at the corners with a opposed), as Section
    5.4 states for eta = 1."""
    n = 201
    speed, drift = hi.zermelo_fields(n, 1.0, math.pi / 4)
    d = drift.reshape(-1, 2).astype(np.float64)
    b = np.hypot(d[:, 0], d[:, 1])
    c = speed.astype(np.float64)
    X1, X2 = hi.mesh(n)
    r = np.hypot(X1, X2).reshape(-1)
    off = r > 0
    np.testing.assert_allclose(b[off] * (1 + r[off] ** 2), 1.0, rtol=2e-6)
    np.testing.assert_allclose(c * (1 + r ** 2), 0.5, rtol=2e-6)
    assert abs((b + c).max() - 1.5) < 0.02           # next to the origin
    assert abs((b - c)[off].min() - 1.0 / 6.0) < 1e-6   # the corners, |x|^2 = 2 (b(0) = 0 is excluded)


def test_table0_rows_have_the_stated_dynamics():
    n = 50
    a = hi.table0_instance("A", 0.0, n=n)
    assert (a.speed == 0).all()
    np.testing.assert_array_equal(a.drift.reshape(-1, 2), np.tile([1.0, 0.0], (n * n, 1)).astype(np.float32))
    assert abs(a.h - 0.5 * 2.0 / (n - 1)) < 1e-15 and a.lam == 0.0
    b = hi.table0_instance("Bchi", 1e-2, n=n)
    X1, _ = hi.mesh(n)
    np.testing.assert_array_equal(b.speed, np.where(X1 >= 0, 2.0, 1.0).astype(np.float32).reshape(-1))
    assert abs(b.sigma - 0.1) < 1e-15                  # sqrt(eps), eps = 1e-2
