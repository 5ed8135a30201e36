"""hjb_residual_noalloc: the FP64 residual for callers that cannot allocate device
memory (a latency-bound loop, or a process whose device memory belongs to another
allocator).  Called through the C ABI with caller-owned device buffers, it must
agree with hjb_residual on the same value field, call after call."""
import ctypes

import numpy as np
import pytest

import hjb_inputs as hi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_residual_noalloc_matches_hjb_residual_two_calls():
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the -m gpu tests")
    from paper_1502_01629_gb300 import Problem, build
    from paper_1502_01629_gb300._lib import HJB_OK, HJB_ERR_INVALID_ARG, lib
    build.build()
    dev = torch.device("cuda", 0)
    inst = hi.patchy_1025(0.02, n=129, coarse_n=17)
    speed = torch.from_numpy(inst.speed).to(dev)
    mask = torch.from_numpy(inst.mask).to(dev)
    ctrl = torch.from_numpy(np.ascontiguousarray(inst.controls, np.float64)).to(dev)
    out = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    with Problem.from_instance(inst, stream=stream) as P:
        for seed in (3, 4):                       # two calls in a row
            u = hi.random_values(inst.n, seed, 0.0, 1.0, inst.mask)
            u = u.astype(np.float32).astype(np.float64)   # hjb_residual widens FP32 values
            P.set_value(u)
            ref = P.residual()
            ud = torch.from_numpy(u).to(dev)
            rc = lib().hjb_residual_noalloc(ctypes.byref(P.desc), speed.data_ptr(), mask.data_ptr(),
                                            None, ctrl.data_ptr(), ud.data_ptr(), out.data_ptr(),
                                            ctypes.c_void_p(stream.cuda_stream))
            assert rc == HJB_OK
            torch.cuda.synchronize()
            got = float(out.item())
            assert ref > 0
            assert abs(got - ref) <= 1e-14 * max(1.0, ref), (got, ref)
    # a grid larger than the fixed scratch is refused before any device work
    big = type(P.desc)()
    ctypes.memmove(ctypes.byref(big), ctypes.byref(P.desc), ctypes.sizeof(big))
    big.n = 8193
    rc = lib().hjb_residual_noalloc(ctypes.byref(big), speed.data_ptr(), mask.data_ptr(), None,
                                    ctrl.data_ptr(), out.data_ptr(), out.data_ptr(), None)
    assert rc == HJB_ERR_INVALID_ARG
