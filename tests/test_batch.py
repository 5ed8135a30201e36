"""The batched solve (many independent problems through one set of launches):
every instance must meet the same gates against the FP64 oracle as a problem
solved alone -- FP32 values within 1e-5 * max(1, |u|), 1e-10 after the FP64
polish, u_hat within the coarse tolerance, labels bit-exact given a* -- and
invalid batches are rejected on the host."""
import ctypes

import numpy as np
import pytest

import hjb_inputs as hi
import oracle


def _small_batch():
    # the many-instance recipe at test sizes: mixed n, sigma, lambda, targets
    return [hi.batched_instance(1000 + k, n=n) for k, n in enumerate((33, 41, 49, 57, 65, 45))]


# ----------------------------------------------------------------- host only

def _create(L, insts, **kw):
    arr = (L.BatchInst * len(insts))()
    for i, x in enumerate(insts):
        arr[i].n, arr[i].coarse_n, arr[i].n_patches, arr[i].reserved = x.n, x.coarse_n, x.n_patches, 0
        arr[i].h, arr[i].lam, arr[i].sigma = x.h, x.lam, x.sigma
        for k, v in kw.get("inst", {}).items():
            if i == kw.get("at", 0):
                setattr(arr[i], k, v)
    d = L.BatchDesc()
    d.n_controls, d.scheme, d.tile_shape, d.tile_waves, d.tile_period, d.schedule = 32, 3, -1, 0, 2, 0
    d.cost, d.band_width = 1.0, 1.0
    for k, v in kw.get("desc", {}).items():
        setattr(d, k, v)
    speed = np.concatenate([x.speed for x in insts]).astype(np.float32)
    mask = np.concatenate([x.mask for x in insts]).astype(np.uint8)
    if "speed_at" in kw:
        speed[kw["speed_at"]] = np.nan
    if "mask_at" in kw:
        mask[kw["mask_at"]] = 7
    ctr = np.ascontiguousarray(insts[0].controls, np.float64)
    h = ctypes.c_void_p()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    return L.lib().hjb_batch_create(ctypes.byref(d), kw.get("count", len(insts)),
                                    ctypes.cast(arr, ctypes.c_void_p), p(speed), p(mask), None,
                                    p(ctr), None, ctypes.byref(h))


@pytest.mark.parametrize("bad", [
    dict(count=0), dict(desc=dict(n_controls=0)), dict(desc=dict(scheme=5)),
    dict(desc=dict(tile_shape=4)), dict(desc=dict(schedule=2)), dict(desc=dict(cost=0.0)),
    dict(inst=dict(n=5)), dict(inst=dict(coarse_n=7), at=1), dict(inst=dict(lam=0.0), at=2),
    dict(inst=dict(sigma=-1.0)), dict(inst=dict(n_patches=0), at=3), dict(inst=dict(reserved=1)),
])
def test_invalid_batches_are_rejected_on_host(bad):
    from paper_1502_01629_gb300 import build
    build.build()
    from paper_1502_01629_gb300 import _lib as L
    rc = _create(L, _small_batch(), **bad)
    assert rc == L.HJB_ERR_INVALID_ARG
    assert L.lib().hjb_last_error()


# ----------------------------------------------------------------------- GPU

@pytest.mark.gpu
@pytest.mark.parametrize("bad", [dict(speed_at=100), dict(mask_at=5000)])
def test_invalid_node_arrays_are_rejected_on_the_device(bad):
    """The concatenated per-node arrays are checked on the device after the
    upload; a bad entry is refused with HJB_ERR_INVALID_ARG."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the -m gpu tests")
    from paper_1502_01629_gb300 import build
    build.build()
    from paper_1502_01629_gb300 import _lib as L
    rc = _create(L, _small_batch(), **bad)
    assert rc == L.HJB_ERR_INVALID_ARG
    assert b"instance" in L.lib().hjb_last_error()


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the -m gpu tests")
    from paper_1502_01629_gb300 import build
    build.build()
    import paper_1502_01629_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def refs():
    """Per-instance oracle results: fixed point, coarse pre-computation."""
    out = []
    for inst in _small_batch():
        O = oracle.Problem.from_instance(inst)
        u, _, _ = O.solve(scheme=3, tol=1e-14)
        pre = oracle.patchy_precompute(inst, tol_c=1e-10)
        out.append((inst, O, u, pre))
    return out


@pytest.mark.gpu
def test_batch_matches_oracle_per_instance(gpu, refs):
    insts = [r[0] for r in refs]
    with gpu.Batch.from_instances(insts) as B:
        st, res = B.solve(tol_c=1e-6, tol32=3e-7, tol64=0.0)
        for i, (inst, O, u_ref, pre) in enumerate(refs):
            scale = max(1.0, np.abs(u_ref).max())
            assert np.abs(B.get_value(i) - u_ref).max() <= 1e-5 * scale, i
        st, res = B.solve(tol_c=1e-6, tol32=3e-7, tol64=1e-12)
        assert (res <= 1e-12).all(), res
        assert st["residual"] <= 1e-12
        for i, (inst, O, u_ref, pre) in enumerate(refs):
            u = B.get_value(i)
            np.testing.assert_allclose(u, u_ref, rtol=0, atol=1e-10)
            assert abs(O.residual(u) - res[i]) <= 1e-13


@pytest.mark.gpu
def test_batch_precomputation_matches_oracle(gpu, refs):
    """u_hat within the coarse tolerance, a* a valid minimiser, labels bit-exact
    given the batch's own a* (the oracle's transport rule applied to it)."""
    insts = [r[0] for r in refs]
    with gpu.Batch.from_instances(insts) as B:
        B.solve(tol_c=1e-6, tol32=3e-7, tol64=0.0)
        for i, (inst, O, u_ref, pre) in enumerate(refs):
            bc = pre["coarse"].beta
            uh = B.get_uhat(i)
            assert np.abs(uh - pre["uhat"]).max() <= 2e-6 / (1 - bc) + 1e-5, i
            a = B.get_feedback(i)
            free = np.flatnonzero(inst.mask == 0)
            assert (a[inst.mask != 0] == 255).all()
            vals = O.synthesis_values(pre["uhat"], free)
            chosen = vals[np.arange(free.size), a[free]]
            assert (chosen - vals.min(axis=1) <= 4e-5).all(), i
            succ = O.successors(a)
            lab = O.labels(succ, inst.sector, inst.n_patches)
            np.testing.assert_array_equal(B.get_labels(i), lab)


@pytest.mark.gpu
def test_batch_jacobi_comparator(gpu, refs):
    insts = [r[0] for r in refs]
    with gpu.Batch.from_instances(insts) as B:
        st, res = B.solve_full(tol32=2.5e-7, tol64=1e-6)
        assert (res <= 1e-6).all(), res
        for i, (inst, O, u_ref, pre) in enumerate(refs):
            u = B.get_value(i)
            assert np.abs(u - u_ref).max() <= 1e-5 * max(1.0, np.abs(u_ref).max()), i
            assert abs(O.residual(u) - res[i]) <= 1e-13


@pytest.mark.gpu
def test_batch_autotune_then_solve(gpu, refs):
    insts = [r[0] for r in refs]
    with gpu.Batch.from_instances(insts) as B:
        t = B.autotune(tol_c=1e-6, tol32=3e-7)
        assert t["tile_shape"] in (0, 1, 2) and t["tile_waves"] in (1, 2)
        assert all(v > 0 for v in t["ms"].values())
        st, res = B.solve(tol_c=1e-6, tol32=3e-7, tol64=1e-12)
        for i, (inst, O, u_ref, pre) in enumerate(refs):
            np.testing.assert_allclose(B.get_value(i), u_ref, rtol=0, atol=1e-10)


@pytest.mark.gpu
@pytest.mark.parametrize("shape,waves", [(0, 1), (1, 2), (2, 2)])
def test_batch_every_tile_shape(gpu, refs, shape, waves):
    insts = [r[0] for r in refs]
    with gpu.Batch.from_instances(insts, tile_shape=shape, tile_waves=waves) as B:
        st, res = B.solve(tol_c=1e-6, tol32=3e-7, tol64=1e-12)
        for i, (inst, O, u_ref, pre) in enumerate(refs):
            np.testing.assert_allclose(B.get_value(i), u_ref, rtol=0, atol=1e-10)
