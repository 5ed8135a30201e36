"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Inputs come from ``hjb_inputs`` (seeded, synthetic, shaped like the paper's 2-D
tests); expected values come from ``oracle`` only.  Tolerances:
  * FP64 operator / solutions: 1e-12 per application, 1e-10 after the FP64
    polish (the FP64 gate);
  * FP32 operator: 2e-6 (a handful of FP32 roundings on values <= ~1);
  * FP32 solutions: 1e-5 * max(1, |u|_inf) (the FP32 gate);
  * integer outputs (successors, labels) bit-exact given the same a*;
  * argmins: exact where the oracle's best candidate is unique by more than
    the arithmetic's error, otherwise the chosen candidate must be within it.
"""
import numpy as np
import pytest

import hjb_inputs as hi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the -m gpu tests")
    from paper_1502_01629_gb300 import build
    build.build()


def P_gpu(inst, **kw):
    from paper_1502_01629_gb300 import Problem
    return Problem.from_instance(inst, **kw)


def instance_variants():
    n = 37
    out = []
    out.append(("disc-s0", hi.disc_instance(n, 0.0, n_controls=32, speed=hi.speed_sine(n))))
    out.append(("disc-s005", hi.disc_instance(n, 0.05, n_controls=32, speed=hi.speed_sine(n))))
    inst = hi.disc_instance(101, 0.1, n_controls=33, speed=hi.speed_sine(101), lam=0.7)
    out.append(("n101-na33-s01", inst))
    inst = hi.disc_instance(150, 0.02, n_controls=64, speed=hi.speed_sine(150), lam=2.0)
    out.append(("n150-na64", inst))
    rng = np.random.default_rng(5)
    inst = hi.disc_instance(45, 0.03, n_controls=16, speed=hi.speed_fourier(45, rng))
    inst.drift = rng.uniform(-0.4, 0.4, 2 * 45 * 45).astype(np.float32)
    inst.mask = hi.add_rect_obstacles(45, inst.mask, [(0.3, 0.3, 0.6, 0.5)])
    out.append(("drift-obstacle", inst))
    inst = hi.disc_instance(20, 0.2, n_controls=1, speed=hi.speed_constant(20, 0.3))
    out.append(("na1-bigsigma", inst))
    return out


VARIANTS = instance_variants()


BAND_CASES = {
    "lambda1": lambda: hi.patchy_1025(0.02, n=257, coarse_n=33),
    "lambda0.7-drift": lambda: _drift_case(),
    "no-discount": lambda: hi.zermelo_instance(97, eps=0.01, coarse_n=25),
}


def _drift_case():
    inst = hi.disc_instance(161, 0.05, n_controls=32, speed=hi.speed_sine(161), lam=0.7,
                            coarse_n=21)
    rng = np.random.default_rng(11)
    inst.drift = rng.uniform(-0.3, 0.3, 2 * 161 * 161).astype(np.float32)
    return inst


@pytest.mark.parametrize("case", list(BAND_CASES))
def test_band_keys_bit_exact_given_the_same_uhat(case):
    """Section 4.2 orders the nodes by increasing u_hat; the causal band key of a
    value is an exact comparison with FP64 band edges on both sides, so given the
    same u_hat (the oracle's, rounded to FP32) the keys agree node for node, and
    the ordering groups every band's nodes by patch."""
    inst = BAND_CASES[case]()
    ref = oracle.patchy_precompute(inst, tol_c=1e-9)
    O = ref["fine"]
    u32 = ref["uhat"].astype(np.float32)
    free = np.flatnonzero(inst.mask == 0)
    with P_gpu(inst) as G:
        G.coarse_solve(tol_c=1e-7)
        G.build_patches()
        G.set_uhat(u32)
        keys, order, off = G.get_order()
        np.testing.assert_array_equal(G.get_uhat()[free], u32[free])
    key_or = oracle.band_keys(u32.astype(np.float64), inst.mask, inst.lam, O.h, 1 << 20)
    np.testing.assert_array_equal(keys[free], key_or[free])
    assert (keys[inst.mask != 0] == -1).all()
    kk = keys[order]
    assert np.array_equal(np.sort(order), free)
    for b in range(len(off) - 1):
        assert (kk[off[b]:off[b + 1]] == b).all()
    assert len(off) - 1 == key_or[free].max() + 1


@pytest.mark.parametrize("name,inst", VARIANTS, ids=[v[0] for v in VARIANTS])
@pytest.mark.parametrize("scheme", [3, 2])
def test_operator_parity_fp64(name, inst, scheme):
    """One application of eq. SLscheme3 / SLscheme2 to a seeded random value field."""
    O = oracle.Problem.from_instance(inst)
    u = O.fix_nonfree(hi.random_values(inst.n, 11, 0.0, O.u_max, inst.mask))
    exp, am_o, _ = O.apply(u, scheme)
    with P_gpu(inst) as G:
        got, am_g = G.apply_operator(u, precision=64, scheme=scheme)
    np.testing.assert_allclose(got, exp, rtol=0, atol=1e-12)
    _check_argmin(O, u, scheme, am_g, am_o, inst.mask, 1e-11)


@pytest.mark.parametrize("name,inst", VARIANTS, ids=[v[0] for v in VARIANTS])
def test_operator_parity_fp32(name, inst):
    O = oracle.Problem.from_instance(inst)
    u = O.fix_nonfree(hi.random_values(inst.n, 12, 0.0, O.u_max, inst.mask))
    u = u.astype(np.float32).astype(np.float64)        # the FP32 path sees FP32 inputs
    exp, am_o, _ = O.apply(u, 3)
    with P_gpu(inst) as G:
        got, am_g = G.apply_operator(u, precision=32, scheme=3)
    np.testing.assert_allclose(got, exp, rtol=0, atol=2e-6 * max(1.0, O.u_max))
    _check_argmin(O, u, 3, am_g, am_o, inst.mask, 4e-6 * max(1.0, O.u_max))


def _check_argmin(O, u, scheme, am_g, am_o, mask, tol):
    free = np.flatnonzero(mask == 0)
    assert (am_g[mask != 0] == -1).all()
    diff = free[am_g[free] != am_o[free]]
    if diff.size:
        vals = O.node_candidates(u, diff, scheme)
        best = vals.min(axis=1)
        chosen = vals[np.arange(diff.size), am_g[diff]]
        assert (chosen - best <= tol).all(), (chosen - best).max()
    assert diff.size <= max(3, free.size // 100)


def test_plain_full_grid_fp64_matches_oracle():
    """The plain FP64 workload (101^2, sigma = 0.05, 32 controls): Jacobi from u = 0
    to a sup-increment of 1e-8, then to 1e-13 for the 1e-10 gate."""
    inst = hi.plain_101()
    O = oracle.Problem.from_instance(inst)
    u_ref, _, _ = O.solve(scheme=3, tol=1e-14)
    u_jac, sweeps_or, _ = O.solve(scheme=3, method="jacobi", tol=1e-8)
    with P_gpu(inst) as G:
        st = G.solve_full(precision=64, tol=1e-8, tol64=0.0)
        assert abs(st["sweeps"] - sweeps_or) <= 8          # checked every 8 sweeps
        u8 = G.get_value()
        assert np.abs(u8 - u_ref).max() <= 1e-8 / (1.0 - O.beta)
        st = G.solve_full(precision=64, tol=1e-13, tol64=0.0)
        u = G.get_value()
        assert st["residual"] <= 1e-13
    np.testing.assert_allclose(u, u_ref, rtol=0, atol=1e-10)


@pytest.mark.parametrize("sigma", [0.0, 0.02, 0.1])
def test_full_grid_fp32_then_fp64(sigma):
    inst = hi.patchy_1025(sigma, n=129, coarse_n=17)
    O = oracle.Problem.from_instance(inst)
    u_ref, _, _ = O.solve(scheme=3, tol=1e-14)
    with P_gpu(inst) as G:
        st = G.solve_full(precision=32, tol=3e-7, tol64=0.0)
        u32 = G.get_value()
        assert np.abs(u32 - u_ref).max() <= 1e-5 * max(1.0, np.abs(u_ref).max())
        st = G.solve_full(precision=32, tol=3e-7, tol64=1e-13)
        assert st["residual"] <= 1e-12
        u = G.get_value()
    np.testing.assert_allclose(u, u_ref, rtol=0, atol=1e-10)


def _oracle_pipeline(inst, tol_c=1e-9):
    return oracle.patchy_precompute(inst, tol_c=tol_c)


@pytest.mark.parametrize("sigma", [0.0, 0.02, 0.1])
def test_patchy_pipeline_small(sigma):
    """Coarse solve, u_hat, a*, labels, ordering and the band-ordered solve on the
    patchy workload at 257^2 (coarse 33^2), against the oracle."""
    inst = hi.patchy_1025(sigma, n=257, coarse_n=33)
    O = oracle.Problem.from_instance(inst)
    ref = _oracle_pipeline(inst)
    with P_gpu(inst) as G:
        cs = G.coarse_solve(tol_c=1e-7)
        uc = G.get_coarse_value()
        # FP32 coarse iteration stopped at 1e-7: error <= 1e-7 / (1 - beta_c) + rounding
        bc = ref["coarse"].beta
        assert np.abs(uc - ref["uc"]).max() <= 2e-7 / (1 - bc) + 1e-5
        G.build_patches()
        uh = G.get_uhat()
        assert np.abs(uh - ref["uhat"]).max() <= 2e-7 / (1 - bc) + 1e-5
        # synthesis: the chosen control is a minimiser of the oracle's objective up
        # to the difference of the two u_hat
        a = G.get_feedback()
        free = np.flatnonzero(inst.mask == 0)
        assert (a[inst.mask != 0] == 255).all()
        diff = free[a[free] != ref["a"][free]]
        assert diff.size <= free.size // 50
        if diff.size:
            vals = O.synthesis_values(ref["uhat"], diff)
            chosen = vals[np.arange(diff.size), a[diff]]
            assert (chosen - vals.min(axis=1) <= 4e-5).all()
        # labels bit-exact given the oracle's a*
        G.set_feedback(ref["a"])
        np.testing.assert_array_equal(G.get_successors(), ref["succ"])
        lab = G.get_labels()
        np.testing.assert_array_equal(lab, ref["labels"])
        keys, order, off = G.get_order()
        # ordering: a permutation of the free nodes, grouped by nondecreasing band
        assert np.array_equal(np.sort(order), free)
        kk = keys[order]
        assert (np.diff(kk) >= 0).all()
        for b in range(len(off) - 1):
            assert (kk[off[b]:off[b + 1]] == b).all()
        key_or = oracle.band_keys(ref["uhat"], inst.mask, inst.lam, O.h, 1 << 20)
        assert (np.abs(keys[free] - key_or[free]) <= 1).all()
        assert (keys[free] == key_or[free]).mean() > 0.99
        # within a band the nodes are grouped by patch
        for b in range(0, len(off) - 1, max(1, (len(off) - 1) // 20)):
            seg = lab[order[off[b]:off[b + 1]]]
            assert (np.diff(seg.astype(int)) >= 0).all()
        # solve: FP32 phase, then FP64 polish
        st = G.solve_patches(tol32=3e-7, tol64=0.0)
        u32 = G.get_value()
        u_ref, _, _ = O.solve(scheme=3, order=np.argsort(ref["uhat"], kind="stable"), tol=1e-14)
        assert np.abs(u32 - u_ref).max() <= 1e-5 * max(1.0, np.abs(u_ref).max())
        st = G.solve_patches(tol32=3e-7, tol64=1e-12)
        assert st["residual"] <= 1e-12
        u = G.get_value()
    np.testing.assert_allclose(u, u_ref, rtol=0, atol=1e-10)


def test_paper_mode_case_a_on_gpu():
    """Section 5.1, Case A (b = (1,0) read with inflow on the left, eps = 0,
    undiscounted, exit through the boundary): the solution is u = x1 + 1."""
    n = 50
    dx = 2.0 / (n - 1)
    mask = hi.square_boundary_target(n)
    drift = np.zeros((n * n, 2), np.float32)
    drift[:, 0] = -1.0
    inst = hi.Instance(n=n, controls=np.array([[1.0, 0.0]]), speed=hi.speed_constant(n, 0.0),
                       mask=mask, sector=hi.sectors_square_sides(n, mask), h=dx / 2, lam=0.0,
                       sigma=0.0, drift=drift.reshape(-1), n_patches=4)
    with P_gpu(inst) as G:
        G.solve_full(precision=64, tol=1e-13, tol64=0.0)
        u = G.get_value()
    x1 = hi.mesh(n)[0].ravel()
    free = mask == 0
    np.testing.assert_allclose(u[free], x1[free] + 1.0, rtol=0, atol=1e-10)


def test_edge_cases_tiny_and_all_target():
    # smallest grid: 3x3 with one free node
    n = 3
    mask = np.ones(9, np.uint8)
    mask[4] = 0
    inst = hi.Instance(n=n, controls=hi.control_set(8), speed=hi.speed_constant(n), mask=mask,
                       sector=np.where(mask == 1, 0, -1).astype(np.int8), sigma=0.3, lam=1.0,
                       coarse_n=3, n_patches=1)
    O = oracle.Problem.from_instance(inst)
    u_ref, _, _ = O.solve(tol=1e-15)
    with P_gpu(inst) as G:
        G.solve_full(precision=64, tol=1e-14, tol64=0.0)
        np.testing.assert_allclose(G.get_value(), u_ref, atol=1e-12)
        G.coarse_solve(tol_c=1e-7)
        G.build_patches()
        G.solve_patches(tol32=1e-7, tol64=1e-13)
        np.testing.assert_allclose(G.get_value(), u_ref, atol=1e-10)
    # every node a target: nothing to update
    inst = hi.Instance(n=5, controls=hi.control_set(4), speed=hi.speed_constant(5),
                       mask=np.ones(25, np.uint8), sector=np.zeros(25, np.int8), coarse_n=3)
    with P_gpu(inst) as G:
        G.coarse_solve()
        G.build_patches()
        G.solve_patches(tol32=1e-7, tol64=1e-12)
        assert (G.get_value() == 0).all()
        G.solve_full(precision=32, tol=1e-7, tol64=1e-12)


def test_warm_start_and_state_errors():
    from paper_1502_01629_gb300 import HJBError
    inst = hi.patchy_1025(0.02, n=65, coarse_n=17)
    O = oracle.Problem.from_instance(inst)
    u_ref, _, _ = O.solve(tol=1e-14)
    with P_gpu(inst) as G:
        with pytest.raises(HJBError):
            G.build_patches()                   # coarse_solve has not run
        with pytest.raises(HJBError):
            G.solve_patches()
        G.coarse_solve()
        G.build_patches()
        # resume from a perturbed copy of the solution: same fixed point
        G.set_value(u_ref + 0.01 * (inst.mask == 0))
        G.solve_patches(tol32=1e-7, tol64=1e-13)
        np.testing.assert_allclose(G.get_value(), u_ref, atol=1e-10)
        assert G.residual() <= 1e-12


@pytest.mark.parametrize("name,inst", VARIANTS[:5], ids=[v[0] for v in VARIANTS[:5]])
def test_fp64_residual_equals_unscreened(name, inst):
    """hjb_residual screens the controls in FP32 and evaluates only the survivors
    in FP64; the result must equal the plain FP64 sup-residual of eq. SLscheme2
    (one full FP64 operator application), on a random field and near a solution."""
    O = oracle.Problem.from_instance(inst)
    with P_gpu(inst) as G:
        for u in (O.fix_nonfree(hi.random_values(inst.n, 21, 0.0, O.u_max, inst.mask)),
                  O.solve(scheme=3, tol=1e-7, max_sweeps=4000)[0]):
            u = u.astype(np.float32).astype(np.float64)
            G.set_value(u)
            r_scr = G.residual()
            tu, _ = G.apply_operator(u, precision=64, scheme=2)
            free = inst.mask == 0
            r_full = np.abs(tu - u)[free].max()
            assert abs(r_scr - r_full) <= 1e-15 * max(1.0, r_full), (r_scr, r_full)
            assert abs(r_scr - O.residual(u)) <= 1e-13


SCHEDULES = [dict(schedule=0, tile_shape=0), dict(schedule=0, tile_shape=1),
             dict(schedule=0, tile_shape=2), dict(schedule=0, tile_shape=0, tile_waves=8, tile_period=4),
             dict(schedule=0, resort_passes=1), dict(schedule=0, local_sweeps=2),
             dict(schedule=1, band_group=1), dict(schedule=1, band_group=4, wave_warps=1024),
             dict(schedule=2, tile_waves=8, tile_period=4),
             dict(schedule=0, visit=1), dict(schedule=0, visit=2, local_sweeps=2),
             dict(schedule=0, tile_shape=1, visit=2),
             dict(schedule=3), dict(schedule=3, tile_shape=1), dict(schedule=3, visit=2, local_sweeps=3),
             dict(schedule=3, tile_shape=2),
             dict(schedule=0, visit=3), dict(schedule=0, tile_shape=0, visit=3), dict(schedule=3, visit=3),
             dict(schedule=0, visit=4), dict(schedule=0, tile_shape=0, visit=4), dict(schedule=3, visit=4)]


@pytest.mark.parametrize("sched", SCHEDULES, ids=[str(s) for s in SCHEDULES])
@pytest.mark.parametrize("sigma", [0.0, 0.05])
def test_every_patch_schedule_reaches_the_oracle_fixed_point(sched, sigma):
    """The fixed point does not depend on the visiting order (Section 4.2): every
    schedule -- warp tiles of each shape, block tiles, band waves, re-sorting,
    extra local sweeps -- must reach the oracle's solution within the gates."""
    inst = hi.patchy_1025(sigma, n=129, coarse_n=17)
    O = oracle.Problem.from_instance(inst)
    u_ref, _, _ = O.solve(scheme=3, tol=1e-14)
    with P_gpu(inst, **sched) as G:
        G.coarse_solve(tol_c=1e-7)
        G.build_patches()
        G.solve_patches(tol32=3e-7, tol64=0.0)
        u32 = G.get_value()
        assert np.abs(u32 - u_ref).max() <= 1e-5 * max(1.0, np.abs(u_ref).max())
        st = G.solve_patches(tol32=3e-7, tol64=1e-12)
        assert st["residual"] <= 1e-12
        np.testing.assert_allclose(G.get_value(), u_ref, rtol=0, atol=1e-10)


@pytest.mark.parametrize("visit", [0, 1, 3])
def test_large_recipe_matches_oracle(visit):
    """The large workload's recipe (random Fourier speed, 64 controls, six
    rectangular obstacles held at the obstacle value, sigma = 0.01, 64 sectors)
    at 129^2 with a 33^2 coarse grid: the patchy solve with the automatic tile
    schedule (8x8 tiles: more than 32 controls) meets the FP32 gate, then the
    FP64 gate after polishing -- with the automatic visits (two nodes at a time:
    the 64 controls are closed under quarter turns), one node at a time, and two
    nodes at a time by request."""
    inst = hi.large_instance(n=129, coarse_n=33)
    O = oracle.Problem.from_instance(inst)
    u_ref, _, _ = O.solve(scheme=3, tol=1e-13)
    scale = max(1.0, np.abs(u_ref).max())
    with P_gpu(inst, visit=visit) as G:
        G.coarse_solve(tol_c=1e-7)
        G.build_patches()
        G.solve_patches(tol32=3e-7, tol64=0.0)
        u32 = G.get_value()
        assert np.abs(u32 - u_ref).max() <= 1e-5 * scale
        st = G.solve_patches(tol32=3e-7, tol64=1e-12)
        assert st["residual"] <= 1e-12
        np.testing.assert_allclose(G.get_value(), u_ref, rtol=0, atol=1e-10)
        u = G.get_value()
    assert np.all(u[inst.mask == hi.MASK_TARGET] == 0.0)
    # obstacle nodes hold l/lambda + h l (obstacles as a penalty: never updated, the largest value); the two sides round the formula
    # differently in the last place
    np.testing.assert_allclose(u[inst.mask == hi.MASK_OBSTACLE], O.u_max, rtol=0, atol=1e-12)


def test_warm_fp32_retry_reaches_the_fp64_tolerance():
    """A loose FP32 tolerance leaves the FP64 residual above tol64; the solver
    then continues in FP32 from the current value with tighter tolerances
    before any FP64 pass.  The result must still satisfy the FP64 residual
    bound and the FP32 value gate against the oracle."""
    inst = hi.patchy_1025(0.02, n=257, coarse_n=33)
    O = oracle.Problem.from_instance(inst)
    u_ref, _, _ = O.solve(scheme=3, tol=1e-12)
    with P_gpu(inst) as G:
        G.coarse_solve(tol_c=1e-7)
        G.build_patches()
        st = G.solve_patches(tol32=1e-4, tol64=1e-6)
        assert st["residual"] <= 1e-6
        assert st["residual_evals"] >= 2          # the first check failed
        u = G.get_value()
        assert np.abs(u - u_ref).max() <= 1e-5 * max(1.0, np.abs(u_ref).max())
        # the oracle's residual of the returned value agrees with the solver's
        assert abs(O.residual(u) - st["residual"]) <= 1e-12


def test_large_workload_full_size_sampled():
    """The 4097^2 large workload as the benchmark runs it (FP32 passes, FP64
    residual <= 1e-6): too large for a full oracle solve, so the FP64 oracle
    evaluates the scheme (eq. SLscheme2) at 3000 sampled free nodes -- random
    ones plus nodes next to obstacles, the target and the domain edge -- from
    the returned value: every sampled |T u - u| must lie within the residual
    the solver reports, and the value must respect the bounds 0 <= u <= u_max."""
    inst = hi.large_instance()
    n = inst.n
    with P_gpu(inst) as G:
        G.coarse_solve(tol_c=1e-6)
        G.build_patches()
        st = G.solve_patches(tol32=5e-7, tol64=1e-6)
        u = G.get_value()
    assert st["residual"] <= 1e-6
    O = oracle.Problem.from_instance(inst)
    m = inst.mask.reshape(n, n)
    free = m == hi.MASK_FREE
    near = np.zeros_like(free)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            near |= np.roll(np.roll(m != hi.MASK_FREE, dy, 0), dx, 1)
    near[0, :] = near[-1, :] = near[:, 0] = near[:, -1] = True
    rng = np.random.default_rng(11)
    special = np.flatnonzero((near & free).reshape(-1))
    pick = np.concatenate([rng.choice(np.flatnonzero(free.reshape(-1)), 2000, replace=False),
                           rng.choice(special, 1000, replace=False)])
    worst = 0.0
    for k in pick:
        v, _ = O.node_update(u, int(k), scheme=2)
        worst = max(worst, abs(v - u[k]))
    assert worst <= st["residual"] * (1 + 1e-9) + 1e-15, (worst, st["residual"])
    assert u.min() >= 0.0 and u.max() <= O.u_max * (1 + 1e-12)
    # obstacle nodes hold l/lambda + h l (obstacles as a penalty: never updated, the largest value); the two sides round the formula
    # differently in the last place
    np.testing.assert_allclose(u[inst.mask == hi.MASK_OBSTACLE], O.u_max, rtol=0, atol=1e-12)


def test_obstacle_values_stay_exact_in_fp64():
    """Obstacle nodes hold l/lambda + h l; with a lambda whose held value is not
    an FP32 number, promoting the FP32 field must not carry the rounded value
    into the FP64 polish (it would move the FP64 fixed point near obstacles)."""
    inst = hi.warmstart_instance(7001, n=65, coarse_n=33)
    assert (inst.mask == hi.MASK_OBSTACLE).any()
    O = oracle.Problem.from_instance(inst)
    assert float(np.float32(O.u_max)) != O.u_max
    u_ref, _, _ = O.solve(scheme=3, tol=1e-14)
    with P_gpu(inst) as G:
        G.coarse_solve(tol_c=1e-6)
        G.build_patches()
        st = G.solve_patches(tol32=3e-7, tol64=1e-12)
        assert st["residual"] <= 1e-12
        np.testing.assert_allclose(G.get_value(), u_ref, rtol=0, atol=1e-10)


def test_invalid_node_arrays_are_rejected_on_the_device():
    """Per-node inputs are checked on the device right after the upload: each bad
    entry is refused with HJB_ERR_INVALID_ARG and its index in the message."""
    from paper_1502_01629_gb300 import Problem, HJBError
    n = 9
    ctr = hi.control_set(4)
    sp = np.ones(n * n, np.float32)
    mk = np.zeros(n * n, np.uint8)
    cases = []
    s = sp.copy(); s[5] = np.nan; cases.append((dict(speed=s), "speed[5]"))
    s = sp.copy(); s[3] = -1.0; cases.append((dict(speed=s), "speed[3]"))
    s = sp.copy(); s[n * n - 1] = np.inf; cases.append((dict(speed=s), f"speed[{n * n - 1}]"))
    m = mk.copy(); m[7] = 3; cases.append((dict(mask=m), "mask[7]"))
    m = mk.copy(); m[0] = 1; sec = np.full(n * n, -1, np.int8); sec[0] = 5
    cases.append((dict(mask=m, sector=sec), "sector[0]"))
    dr = np.zeros(2 * n * n, np.float32); dr[4] = np.nan; cases.append((dict(drift=dr), "drift[2]"))
    for kw, where in cases:
        args = dict(speed=sp, mask=mk)
        args.update(kw)
        with pytest.raises(HJBError) as e:
            Problem(n, ctr, args.pop("speed"), args.pop("mask"), args.pop("sector", None), **args)
        assert e.value.code == -1 and where in str(e.value), (where, str(e.value))
    m = mk.copy(); m[7] = 2
    with pytest.raises(HJBError):
        Problem(n, ctr, sp, m, lam=0.0)             # obstacles need a discount
    with Problem(n, ctr, sp, mk) as P:                # a valid one still builds
        assert P.n == n


@pytest.mark.parametrize("sigma", [0.0, 0.02, 0.1])
def test_patchy_1025_full_size_sampled(sigma):
    """The 1025^2 workload exactly as bench.py runs it (its solver settings and
    tolerances): too large for a full oracle solve at test time, so the FP64
    oracle evaluates eq. SLscheme2 at 3000 sampled free nodes (random ones plus
    nodes next to the target and the domain edge) from the returned values of
    both the patchy solve and the plain Jacobi comparator: every sampled
    |T u - u| lies within the residual each reports, both respect
    0 <= u <= u_max, and the two solutions agree within the distance the two
    residuals allow, (r1 + r2) / (1 - beta)."""
    import bench
    inst = hi.patchy_1025(sigma)
    n = inst.n
    O = oracle.Problem.from_instance(inst)
    with P_gpu(inst, **bench.SOLVER_KW) as G:
        G.coarse_solve(tol_c=bench.TOL_C)
        G.build_patches()
        st = G.solve_patches(tol32=bench.TOL32, tol64=bench.TOL64)
        u = G.get_value()
        sf = G.solve_full(precision=32, tol=bench.TOL32, tol64=bench.TOL64)
        v = G.get_value()
    assert st["residual"] <= bench.TOL64 and sf["residual"] <= bench.TOL64
    m = inst.mask.reshape(n, n)
    free = m == hi.MASK_FREE
    near = np.zeros_like(free)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            near |= np.roll(np.roll(m != hi.MASK_FREE, dy, 0), dx, 1)
    near[0, :] = near[-1, :] = near[:, 0] = near[:, -1] = True
    rng = np.random.default_rng(13)
    special = np.flatnonzero((near & free).reshape(-1))
    pick = np.concatenate([rng.choice(np.flatnonzero(free.reshape(-1)), 2000, replace=False),
                           rng.choice(special, 1000, replace=False)])
    for w, res in ((u, st["residual"]), (v, sf["residual"])):
        worst = max(abs(O.node_update(w, int(k), scheme=2)[0] - w[k]) for k in pick)
        assert worst <= res * (1 + 1e-9) + 1e-15, (worst, res)
        assert w.min() >= 0.0 and w.max() <= O.u_max * (1 + 1e-12)
    assert np.abs(u - v).max() <= (st["residual"] + sf["residual"]) / (1.0 - O.beta) + 1e-12


def test_device_pointer_inputs_match_host_inputs():
    """hjb_create_problem_device takes the per-node arrays as device pointers
    (torch CUDA tensors here): same checks, same problem -- the operator gives
    the host-created problem's results bit for bit, the two patchy solves agree
    within what their FP64 residuals allow (the relaxations read neighbours'
    values as they are being updated, so the last bits may differ), and a bad
    entry is refused the same way."""
    from paper_1502_01629_gb300 import Problem, HJBError
    inst = hi.patchy_1025(0.02, n=129, coarse_n=17)
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    sp, mk, sec = t(inst.speed), t(inst.mask), t(inst.sector)
    kw = dict(sigma=inst.sigma, lam=inst.lam, coarse_n=inst.coarse_n, n_patches=inst.n_patches)
    u = oracle.Problem.from_instance(inst).fix_nonfree(hi.random_values(inst.n, 5, 0.0, 1.0, inst.mask))
    with Problem(inst.n, inst.controls, inst.speed, inst.mask, inst.sector, **kw) as H, \
            Problem(inst.n, inst.controls, sp, mk, sec, device_inputs=True, **kw) as D:
        res = []
        for P in (H, D):
            P.coarse_solve(tol_c=1e-6)
            P.build_patches()
            res.append(P.solve_patches(tol32=3e-7, tol64=1e-10)["residual"])
        beta = 1.0 / (1.0 + inst.lam * 2.0 / (inst.n - 1))
        assert np.abs(D.get_value() - H.get_value()).max() <= sum(res) / (1.0 - beta) + 1e-12
        np.testing.assert_array_equal(D.apply_operator(u)[0], H.apply_operator(u)[0])
    bad = sp.clone()
    bad[17] = float("nan")
    with pytest.raises(HJBError) as e:
        Problem(inst.n, inst.controls, bad, mk, sec, device_inputs=True, **kw)
    assert "speed[17]" in str(e.value)


def test_pool_memory_is_reused_and_trimmed():
    """Problems draw device memory from the library's stream-ordered pool: many
    create / destroy cycles do not grow the device's used memory beyond one
    problem's share, and hjb_trim_memory returns the cached blocks."""
    from paper_1502_01629_gb300 import Problem, lib
    inst = hi.patchy_1025(0.0, n=257, coarse_n=33)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(6):
        with Problem.from_instance(inst) as P:
            P.coarse_solve(tol_c=1e-6)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    one = 200 * inst.n * inst.n                      # well above a problem's ~70 B/node
    assert free0 - free1 <= one + (64 << 20), (free0 - free1)
    assert lib().hjb_trim_memory() == 0
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    assert free2 >= free1
