"""hjb_residual_noalloc: the FP64 residual for callers that cannot allocate device
memory (a latency-bound loop, or a process whose device memory belongs to another
allocator).  Called through the C ABI with caller-owned device buffers, it must
agree with hjb_residual on the same value field, call after call, on every form
of the scheme it serves: no diffusion, diffusion, a drift without a discount, and
obstacles."""
import ctypes

import numpy as np
import pytest

import hjb_inputs as hi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    "sigma0": lambda: hi.patchy_1025(0.0, n=129, coarse_n=17),
    "sigma0.02": lambda: hi.patchy_1025(0.02, n=129, coarse_n=17),
    "drift-no-discount": lambda: hi.zermelo_instance(97, eps=0.01),
    "obstacles-64-controls": lambda: hi.large_instance(n=129, coarse_n=17),
}


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the -m gpu tests")
    from paper_1502_01629_gb300 import build
    build.build()


def _call(desc, speed, mask, drift, ctrl_ptr, u, out, stream=None):
    from paper_1502_01629_gb300._lib import lib
    return lib().hjb_residual_noalloc(
        ctypes.byref(desc), speed.data_ptr(), mask.data_ptr(),
        None if drift is None else drift.data_ptr(), ctrl_ptr, u.data_ptr(), out.data_ptr(),
        None if stream is None else ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("case", list(CASES))
def test_residual_noalloc_matches_hjb_residual_two_calls(case):
    _need_gpu()
    from paper_1502_01629_gb300 import Problem
    from paper_1502_01629_gb300._lib import HJB_OK
    dev = torch.device("cuda", 0)
    inst = CASES[case]()
    speed = torch.from_numpy(inst.speed).to(dev)
    mask = torch.from_numpy(inst.mask).to(dev)
    drift = None if inst.drift is None else torch.from_numpy(inst.drift).to(dev)
    ctrl = torch.from_numpy(np.ascontiguousarray(inst.controls, np.float64)).to(dev)
    out = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    with Problem.from_instance(inst, stream=stream) as P:
        for seed in (3, 4):                       # two calls in a row
            u = hi.random_values(inst.n, seed, 0.0, 1.0, inst.mask)
            u = u.astype(np.float32).astype(np.float64)   # hjb_residual widens FP32 values
            P.set_value(u)
            ref = P.residual()
            # the caller's array holds arbitrary values at obstacle nodes: the
            # entry point takes the obstacle value there, as the solver does
            u_call = u.copy()
            u_call[inst.mask == hi.MASK_OBSTACLE] = 7.0
            ud = torch.from_numpy(u_call).to(dev)
            rc = _call(P.desc, speed, mask, drift, ctrl.data_ptr(), ud, out, stream)
            assert rc == HJB_OK
            torch.cuda.synchronize()
            got = float(out.item())
            assert ref > 0
            assert abs(got - ref) <= 1e-14 * max(1.0, ref), (case, seed, got, ref)


def test_residual_noalloc_nan_is_not_hidden():
    _need_gpu()
    from paper_1502_01629_gb300 import Problem
    from paper_1502_01629_gb300._lib import HJB_OK
    dev = torch.device("cuda", 0)
    inst = hi.patchy_1025(0.02, n=129, coarse_n=17)
    speed = torch.from_numpy(inst.speed).to(dev)
    mask = torch.from_numpy(inst.mask).to(dev)
    ctrl = torch.from_numpy(np.ascontiguousarray(inst.controls, np.float64)).to(dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    u = hi.random_values(inst.n, 5, 0.0, 1.0, inst.mask)
    free = np.flatnonzero(inst.mask == hi.MASK_FREE)
    u[free[free.size // 3]] = np.nan
    with Problem.from_instance(inst) as P:
        rc = _call(P.desc, speed, mask, None, ctrl.data_ptr(), torch.from_numpy(u).to(dev), out)
    assert rc == HJB_OK
    torch.cuda.synchronize()
    assert not np.isfinite(float(out.item()))


def test_residual_noalloc_rejections_and_size_limit():
    _need_gpu()
    from paper_1502_01629_gb300 import Problem
    from paper_1502_01629_gb300._lib import HJB_ERR_INVALID_ARG, HJB_OK
    dev = torch.device("cuda", 0)
    inst = hi.patchy_1025(0.02, n=129, coarse_n=17)
    speed = torch.from_numpy(inst.speed).to(dev)
    mask = torch.from_numpy(inst.mask).to(dev)
    ctrl = torch.from_numpy(np.ascontiguousarray(inst.controls, np.float64)).to(dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    u = torch.zeros(inst.n * inst.n, dtype=torch.float64, device=dev)
    with Problem.from_instance(inst) as P:
        desc = P.desc
    # a controls pointer 8 bytes off its 16-byte alignment
    ctrl2 = torch.zeros(2 * inst.n_controls + 2, dtype=torch.float64, device=dev)
    assert _call(desc, speed, mask, None, ctrl2.data_ptr() + 8, u, out) == HJB_ERR_INVALID_ARG
    # the largest accepted grid: ceil(n/32) ceil(n/16) = 181 x 362 = 65522 tiles
    big = type(desc)()
    ctypes.memmove(ctypes.byref(big), ctypes.byref(desc), ctypes.sizeof(big))
    big.n = 5792
    N = big.n * big.n
    bs = torch.ones(N, dtype=torch.float32, device=dev)
    bm = torch.zeros(N, dtype=torch.uint8, device=dev)
    bm[N // 2 + big.n // 2] = hi.MASK_TARGET
    bu = torch.zeros(N, dtype=torch.float64, device=dev)
    assert _call(big, bs, bm, None, ctrl.data_ptr(), bu, out) == HJB_OK
    torch.cuda.synchronize()
    hl = 2.0 / (big.n - 1) * big.cost
    assert abs(float(out.item()) - hl) <= 1e-12     # u = 0: T u - u = h l at every free node
    del bs, bm, bu
    # one node more per side needs 65703 tiles: refused before any device work
    big.n = 5793
    assert _call(big, speed, mask, None, ctrl.data_ptr(), u, out) == HJB_ERR_INVALID_ARG
    big.n = 8193
    assert _call(big, speed, mask, None, ctrl.data_ptr(), u, out) == HJB_ERR_INVALID_ARG
