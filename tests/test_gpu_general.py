"""Parity of the CUDA path with the FP64 oracle on the general problems of
Section 5: sigma(x) per node (degenerate diffusion), the one-dimensional
diffusion sigma(x) a along the control, the running cost l(x) + m(a), the
Zermelo dynamics and the undiscounted exit-time setting.  Inputs from
``hjb_inputs``, expected values from ``oracle`` only; the tolerances are those
of the constant-coefficient parity tests (FP64 operator 1e-12, FP32 operator
2e-6 max(1, U), FP64 solutions 1e-10)."""
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


def _discounted_general(n=45):
    """A discounted disc problem with obstacles and every general term: sigma(x)
    varying smoothly, diffusion along the control, l(x) and m(a)."""
    rng = np.random.default_rng(17)
    inst = hi.disc_instance(n, 0.0, n_controls=24, speed=hi.speed_fourier(n, rng), lam=0.9)
    inst.mask = hi.add_rect_obstacles(n, inst.mask, [(0.35, 0.3, 0.65, 0.55)])
    X1, X2 = hi.mesh(n)
    inst.sigma_field = (0.08 * (1.0 + np.sin(3.0 * X1) * np.cos(2.0 * X2))).astype(np.float32).reshape(-1)
    inst.diffusion = 1
    inst.cost_field = (1.0 + 0.5 * X1 ** 2).astype(np.float32).reshape(-1)
    inst.control_cost = 0.2 * (1.0 + inst.controls[:, 0])
    inst.name = "discounted-general"
    return inst


def general_variants():
    out = []
    for sk in (1, 2, 3):
        for ck in (1, 2, 3):
            out.append((f"l{ck}-s{sk}", hi.general_instance(45, sk, ck)))
    out.append(("degenerate", hi.degenerate_instance(45)))
    out.append(("zermelo", hi.zermelo_instance(45)))
    out.append(("zermelo-eta0", hi.zermelo_instance(45, eta=0.0)))
    # a wide diffusion along the control (several cells) to exercise the projection
    out.append(("wide-along", hi.general_instance(41, 3, 3, eps=0.1, h=0.5 * 2.0 / 40)))
    out.append(("discounted", _discounted_general()))
    return out


VARIANTS = general_variants()


def _u_scale(O):
    return O.u_max if O.lam > 0 else 2.0


def _check_argmin(O, u, scheme, am_g, am_o, mask, tol):
    free = np.flatnonzero(mask == 0)
    assert (am_g[mask != 0] == -1).all()
    diff = free[am_g[free] != am_o[free]]
    if diff.size:
        vals = O.node_candidates(u, diff, scheme)
        chosen = vals[np.arange(diff.size), am_g[diff]]
        assert (chosen - vals.min(axis=1) <= tol).all(), (chosen - vals.min(axis=1)).max()
    assert diff.size <= max(3, free.size // 100)


@pytest.mark.parametrize("name,inst", VARIANTS, ids=[v[0] for v in VARIANTS])
@pytest.mark.parametrize("scheme", [3, 2])
def test_general_operator_parity_fp64(name, inst, scheme):
    O = oracle.Problem.from_instance(inst)
    u = O.fix_nonfree(hi.random_values(inst.n, 21, 0.0, _u_scale(O), inst.mask))
    exp, am_o, _ = O.apply(u, scheme)
    with P_gpu(inst) as G:
        got, am_g = G.apply_operator(u, precision=64, scheme=scheme)
    np.testing.assert_allclose(got, exp, rtol=0, atol=1e-12 * max(1.0, _u_scale(O)))
    _check_argmin(O, u, scheme, am_g, am_o, inst.mask, 1e-11)


@pytest.mark.parametrize("name,inst", VARIANTS, ids=[v[0] for v in VARIANTS])
def test_general_operator_parity_fp32(name, inst):
    O = oracle.Problem.from_instance(inst)
    u = O.fix_nonfree(hi.random_values(inst.n, 22, 0.0, _u_scale(O), inst.mask))
    u = u.astype(np.float32).astype(np.float64)
    exp, am_o, _ = O.apply(u, 3)
    with P_gpu(inst) as G:
        got, am_g = G.apply_operator(u, precision=32, scheme=3)
    U = max(1.0, _u_scale(O))
    np.testing.assert_allclose(got, exp, rtol=0, atol=2e-6 * U)
    _check_argmin(O, u, 3, am_g, am_o, inst.mask, 4e-6 * U)


@pytest.mark.parametrize("sk,ck", [(1, 3), (2, 2), (3, 3)])
def test_general_full_grid_reaches_the_oracle_fixed_point(sk, ck):
    """Plain full-grid iteration (FP32, then FP64 to the residual gate) on the
    undiscounted problems of Section 5.3."""
    inst = hi.general_instance(45, sk, ck)
    O = oracle.Problem.from_instance(inst)
    u_ref, _, _ = O.solve(scheme=3, tol=1e-14)
    with P_gpu(inst) as G:
        st = G.solve_full(precision=32, tol=3e-7, tol64=1e-13)
        assert st["residual"] <= 1e-12
        u = G.get_value()
    assert O.residual(u) <= 1e-12
    np.testing.assert_allclose(u, u_ref, rtol=0, atol=1e-10)


def _pipeline(inst, tol64=1e-12):
    """The patchy pipeline on the GPU against the oracle's pre-computation and
    fixed point; returns the GPU solution."""
    O = oracle.Problem.from_instance(inst)
    ref = oracle.patchy_precompute(inst, tol_c=1e-10)
    with P_gpu(inst) as G:
        G.coarse_solve(tol_c=1e-7)
        uc = G.get_coarse_value()
        scale = max(1.0, np.abs(ref["uc"]).max())
        assert np.abs(uc - ref["uc"]).max() <= 1e-5 * scale
        G.build_patches()
        uh = G.get_uhat()
        assert np.abs(uh - ref["uhat"]).max() <= 1e-5 * scale
        a = G.get_feedback()
        free = np.flatnonzero(inst.mask == 0)
        diff = free[a[free] != ref["a"][free]]
        assert diff.size <= max(3, free.size // 50)
        if diff.size:
            vals = O.synthesis_values(ref["uhat"], diff)
            chosen = vals[np.arange(diff.size), a[diff]]
            assert (chosen - vals.min(axis=1) <= 4e-5 * scale).all()
        G.set_feedback(ref["a"])
        np.testing.assert_array_equal(G.get_successors(), ref["succ"])
        np.testing.assert_array_equal(G.get_labels(), ref["labels"])
        st = G.solve_patches(tol32=3e-7, tol64=tol64)
        assert st["residual"] <= tol64
        u = G.get_value()
    u_ref, _, _ = O.solve(scheme=3, tol=1e-14)
    np.testing.assert_allclose(u, u_ref, rtol=0, atol=1e-10)
    assert O.residual(u) <= 1e-11
    return u


@pytest.mark.parametrize("sk,ck", [(1, 2), (2, 3), (3, 1), (3, 3)])
def test_general_patchy_pipeline(sk, ck):
    _pipeline(hi.general_instance(65, sk, ck, coarse_n=17))


def test_degenerate_patchy_pipeline():
    _pipeline(hi.degenerate_instance(65, coarse_n=17))


def test_zermelo_patchy_pipeline():
    """Dynamics C: the drift is carried to the coarse grid too."""
    _pipeline(hi.zermelo_instance(65, coarse_n=17))


def test_discounted_general_patchy_pipeline():
    inst = _discounted_general(65)
    inst.coarse_n = 17
    inst.n_patches = 16
    _pipeline(inst)


def test_general_terms_are_validated():
    from paper_1502_01629_gb300 import HJBError
    inst = hi.general_instance(33, 2, 3)
    bad = [dict(sigma_field=np.full(33 * 33, -0.1, np.float32)),
           dict(cost_field=np.zeros(33 * 33, np.float32)),
           dict(control_cost=-np.ones(inst.n_controls)),
           dict(diffusion=2)]
    for kw in bad:
        with pytest.raises(HJBError):
            P_gpu(inst, **kw)
