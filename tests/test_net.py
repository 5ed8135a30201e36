"""The learned warm start's network: the FP64 reference (oracle/convnet.py) is
pinned to independent facts on the CPU -- scipy's correlation for the forward
pass, the adjoint identity for the input gradient, finite differences for the
weight and loss gradients -- and the tensor-core layers (through the C ABI) are
compared with it on the GPU.

Tolerances: inputs and weights are rounded to bfloat16 on both sides, so the
GPU and the reference multiply the same numbers; the GPU accumulates in FP32
(at most 432 products per output for the layers, a few thousand pixels per
weight-gradient entry), hence a relative 1e-4 of the output scale."""
import ctypes

import numpy as np
import pytest

from oracle import convnet as cn


def _rng(seed):
    return np.random.default_rng(np.random.PCG64(seed))


# ------------------------------------------------------------ CPU: the pins

def test_bf16_round_known_values():
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 3.0e38, 0.0])
    r = cn.bf16_round(v)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: ties go to the even mantissa (1.0)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2.0 ** -6 and r[3] == -2.5 and r[5] == 0.0
    assert cn.bf16_bits(np.array([1.0]))[0] == 0x3F80


def test_conv3x3_matches_scipy_correlation():
    from scipy.signal import correlate2d
    rng = _rng(1)
    x = rng.standard_normal((2, 9, 11, 3))
    w = rng.standard_normal((4, 9, 3))
    b = rng.standard_normal(4)
    y = cn.conv3x3(x, w, b)
    for bi in range(2):
        for o in range(4):
            ref = np.full((9, 11), b[o])
            for c in range(3):
                ref += correlate2d(x[bi, :, :, c], w[o, :, c].reshape(3, 3), mode="same",
                                   boundary="fill", fillvalue=0.0)
            np.testing.assert_allclose(y[bi, :, :, o], ref, rtol=1e-12, atol=1e-12)
    # identity kernel: the centre tap copies the input
    wid = np.zeros((3, 9, 3))
    for c in range(3):
        wid[c, 4, c] = 1.0
    np.testing.assert_array_equal(cn.conv3x3(x, wid), x)


def test_taps_past_the_image_read_zero():
    rng = _rng(13)
    x = rng.standard_normal((1, 4, 5, 2))
    w = rng.standard_normal((3, 9, 2))
    # dilation 8 > image: only the centre tap sees the image
    np.testing.assert_allclose(cn.conv3x3(x, w, dil=8), np.einsum("bijc,oc->bijo", x, w[:, 4, :]),
                               rtol=1e-12, atol=1e-12)


def test_dilated_conv3x3_is_a_zero_interleaved_5x5_correlation():
    from scipy.signal import correlate2d
    rng = _rng(12)
    x = rng.standard_normal((1, 10, 9, 2))
    w = rng.standard_normal((3, 9, 2))
    y = cn.conv3x3(x, w, dil=2)
    for o in range(3):
        ref = np.zeros((10, 9))
        for c in range(2):
            k5 = np.zeros((5, 5))
            k5[::2, ::2] = w[o, :, c].reshape(3, 3)
            ref += correlate2d(x[0, :, :, c], k5, mode="same", boundary="fill", fillvalue=0.0)
        np.testing.assert_allclose(y[0, :, :, o], ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dil", [1, 3])
def test_dgrad_is_the_adjoint_of_conv3x3(dil):
    rng = _rng(2)
    x = rng.standard_normal((2, 7, 5, 6))
    dy = rng.standard_normal((2, 7, 5, 4))
    w = rng.standard_normal((4, 9, 6))
    lhs = (cn.conv3x3(x, w, dil=dil) * dy).sum()
    rhs = (x * cn.conv3x3_dgrad(dy, w, dil=dil)).sum()
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))


@pytest.mark.parametrize("dil", [1, 2])
def test_wgrad_is_the_gradient_of_the_pairing(dil):
    rng = _rng(3)
    x = rng.standard_normal((2, 6, 8, 3))
    dy = rng.standard_normal((2, 6, 8, 5))
    w = rng.standard_normal((5, 9, 3))
    b = rng.standard_normal(5)
    dw, db = cn.conv3x3_wgrad(x, dy, dil=dil)
    f = lambda ww, bb: (cn.conv3x3(x, ww, bb, dil=dil) * dy).sum()
    base = f(w, b)
    for (o, t, c) in [(0, 0, 0), (4, 8, 2), (2, 4, 1), (1, 3, 0)]:
        e = np.zeros_like(w)
        e[o, t, c] = 1.0
        assert abs((f(w + e, b) - base) - dw[o, t, c]) <= 1e-9 * max(1.0, abs(dw[o, t, c]))
    for o in range(5):
        e = np.zeros(5)
        e[o] = 1.0
        assert abs((f(w, b + e) - base) - db[o]) <= 1e-9 * max(1.0, abs(db[o]))


def test_loss_gradient_finite_differences():
    rng = _rng(4)
    out = rng.standard_normal((1, 4, 5, 48))
    tval = rng.uniform(0, 1, (1, 4, 5))
    tctrl = rng.integers(0, 32, (1, 4, 5))
    free = rng.uniform(size=(1, 4, 5)) < 0.7
    wv, wc = 1.0, 0.3
    lv, lc, g = cn.loss_and_grad(out, tval, tctrl, free, wv, wc)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (0, 1, 2, 5), (0, 3, 4, 32), (0, 2, 1, 17)]:
        o2 = out.copy()
        o2[idx] += h
        lv2, lc2, _ = cn.loss_and_grad(o2, tval, tctrl, free, wv, wc)
        num = ((wv * lv2 + wc * lc2) - (wv * lv + wc * lc)) / h
        assert abs(num - g[idx]) <= 1e-4 * max(1.0, abs(g[idx])), (idx, num, g[idx])
    assert np.all(g[~free] == 0.0)


# ------------------------------------------------------------- GPU parity

@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the -m gpu tests")
    from paper_1502_01629_gb300 import build
    build.build()
    from paper_1502_01629_gb300 import _lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


SHAPES = [(2, 17, 23, 5, 32, 1), (1, 33, 33, 32, 32, 4), (3, 9, 14, 32, 33, 1), (1, 12, 40, 48, 32, 16),
          (2, 11, 13, 16, 48, 3), (1, 5, 7, 3, 7, 2)]


@pytest.mark.gpu
@pytest.mark.parametrize("B,H,W,cin,cout,dil", SHAPES, ids=[str(s) for s in SHAPES])
def test_conv3x3_forward_on_tensor_cores(L, B, H, W, cin, cout, dil):
    rng = _rng(10 + cin + cout)
    x = cn.bf16_round(rng.uniform(-1, 1, (B, H, W, cin)))
    w = rng.standard_normal((cout, 9, cin)) * 0.2
    b = rng.standard_normal(cout) * 0.1
    for relu in (0, 1):
        y = np.empty((B, H, W, cout), np.float32)
        xb = np.ascontiguousarray(cn.bf16_bits(x))
        wf = np.ascontiguousarray(w, np.float32)
        bf = np.ascontiguousarray(b, np.float32)
        rc = L.lib().hjb_conv3x3_forward(B, H, W, cin, cout, dil, _p(xb), _p(wf), _p(bf), relu, _p(y))
        assert rc == 0, L.lib().hjb_last_error()
        ref = cn.conv3x3(x, cn.bf16_round(wf), bf.astype(np.float64), relu=bool(relu), dil=dil)
        np.testing.assert_allclose(y, ref, rtol=0, atol=1e-4 * max(1.0, np.abs(ref).max()))


@pytest.mark.gpu
@pytest.mark.parametrize("B,H,W,cin,cout,dil", SHAPES, ids=[str(s) for s in SHAPES])
def test_conv3x3_dgrad_on_tensor_cores(L, B, H, W, cin, cout, dil):
    rng = _rng(20 + cin + cout)
    dy = cn.bf16_round(rng.standard_normal((B, H, W, cout)))
    w = rng.standard_normal((cout, 9, cin)) * 0.2
    mask = cn.bf16_round(np.maximum(rng.standard_normal((B, H, W, cin)), 0.0))
    dx = np.empty((B, H, W, cin), np.float32)
    wf = np.ascontiguousarray(w, np.float32)
    rc = L.lib().hjb_conv3x3_dgrad(B, H, W, cin, cout, dil, _p(np.ascontiguousarray(cn.bf16_bits(dy))),
                                   _p(wf), _p(np.ascontiguousarray(cn.bf16_bits(mask))), _p(dx))
    assert rc == 0, L.lib().hjb_last_error()
    ref = cn.conv3x3_dgrad(dy, cn.bf16_round(wf), mask, dil=dil)
    np.testing.assert_allclose(dx, ref, rtol=0, atol=1e-4 * max(1.0, np.abs(ref).max()))


@pytest.mark.gpu
@pytest.mark.parametrize("B,H,W,cin,cout,dil", SHAPES[:4], ids=[str(s) for s in SHAPES[:4]])
def test_conv3x3_wgrad(L, B, H, W, cin, cout, dil):
    rng = _rng(30 + cin + cout)
    x = cn.bf16_round(rng.uniform(-1, 1, (B, H, W, cin)))
    dy = cn.bf16_round(rng.standard_normal((B, H, W, cout)) * 0.1)
    dw = np.empty((cout, 9, cin), np.float32)
    db = np.empty(cout, np.float32)
    rc = L.lib().hjb_conv3x3_wgrad(B, H, W, cin, cout, dil, _p(np.ascontiguousarray(cn.bf16_bits(x))),
                                   _p(np.ascontiguousarray(cn.bf16_bits(dy))), _p(dw), _p(db))
    assert rc == 0, L.lib().hjb_last_error()
    rdw, rdb = cn.conv3x3_wgrad(x, dy, dil=dil)
    np.testing.assert_allclose(dw, rdw, rtol=0, atol=1e-4 * max(1.0, np.abs(rdw).max()))
    np.testing.assert_allclose(db, rdb, rtol=0, atol=1e-4 * max(1.0, np.abs(rdb).max()))


@pytest.mark.gpu
def test_network_training_step_matches_reference_gradients(L):
    """One training step from known parameters: the updated parameters equal a
    reference Adam step on the gradients the FP64 reference computes through the
    whole network (forward of all six layers, loss, backward)."""
    import torch
    from paper_1502_01629_gb300 import Net, NET_DIL
    rng = _rng(40)
    B, H, W = 2, 13, 17
    net = Net(max_batch=B, height=H, width=W)
    params = net.init_params(seed=7)
    net.set_params(params)
    x = cn.bf16_round(np.concatenate([rng.uniform(0, 1, (B, H, W, 5)), np.zeros((B, H, W, 11))], axis=-1))
    tval = rng.uniform(0, 1, (B, H, W)).astype(np.float32)
    tctrl = rng.integers(0, 32, (B, H, W)).astype(np.uint8)
    free = (rng.uniform(size=(B, H, W)) < 0.8).astype(np.uint8)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    xd = dev(cn.bf16_bits(x).view(np.int16))
    lr = 1e-3
    loss = net.train_step(xd, dev(tval), dev(tctrl), dev(free), int(free.sum()), lr=lr, w_value=1.0, w_ctrl=0.1)
    new = net.get_params()
    # FP64 reference of the same step (activations rounded to bf16 as the GPU stores them)
    layers = net.unpack(params)
    acts = [x]
    h = x
    for li, (w, b) in enumerate(layers):
        wq = cn.bf16_round(w)
        if li < 5:
            h = cn.bf16_round(cn.conv3x3(h, wq, b, relu=True, dil=NET_DIL[li]))
            acts.append(h)
        else:
            out = cn.conv3x3(h, wq, b, dil=NET_DIL[li])
    lv, lc, g = cn.loss_and_grad(np.concatenate([out, np.zeros(out.shape[:3] + (15,))], -1), tval, tctrl,
                                 free, 1.0, 0.1)
    assert abs(loss[0] - lv) <= 1e-3 * max(1.0, lv) and abs(loss[1] - lc) <= 1e-3 * max(1.0, lc)
    dz = cn.bf16_round(g[..., :33])
    grads = [None] * 6
    mags = [None] * 6
    for li in range(5, -1, -1):
        w, b = layers[li]
        grads[li] = cn.conv3x3_wgrad(acts[li], dz, dil=NET_DIL[li])
        # sum_p |a_p| |dz_p| of every gradient entry: the scale of its rounding error
        mags[li] = cn.conv3x3_wgrad(np.abs(acts[li]), np.abs(dz), dil=NET_DIL[li])
        if li > 0:
            dz = cn.bf16_round(cn.conv3x3_dgrad(dz, cn.bf16_round(w), acts[li], dil=NET_DIL[li]))
    ref_grad = net.pack([(gw, gb) for gw, gb in grads])
    mag = net.pack([(mw, mb) for mw, mb in mags])
    got = net.get_grads()
    # element by element: an activation or gradient stored in BF16 may round the
    # other way on the GPU (FP32 sums in another order), one BF16 ulp = 2^-8
    # relative; a few such flips along the layers give at most 2^-6 of the
    # magnitude sum of the entry, plus FP32 summation error
    tol = 2.0 ** -6 * mag + 1e-6 * np.abs(ref_grad).max()
    bad = np.abs(got - ref_grad) > tol
    assert not bad.any(), (int(bad.sum()), float(np.abs(got - ref_grad)[bad].max()))
    # first Adam step: update = lr * g / (sqrt(g^2) + eps) with the GPU's own gradient
    ref_new = params - lr * got / (np.abs(got) + 1e-8)
    np.testing.assert_allclose(new, ref_new, rtol=0, atol=2e-6)
    net.close()


@pytest.mark.gpu
def test_network_learns_a_smooth_target(L):
    """A few hundred Adam steps on a fixed batch drive the loss down."""
    import torch
    from paper_1502_01629_gb300 import Net
    rng = _rng(50)
    B, H, W = 4, 33, 33
    net = Net(max_batch=B, height=H, width=W)
    net.set_params(net.init_params(seed=3))
    yy, xx = np.meshgrid(np.linspace(-1, 1, H), np.linspace(-1, 1, W), indexing="ij")
    x = np.zeros((B, H, W, 16))
    x[..., 0] = rng.uniform(0.5, 1.5, (B, 1, 1)) * (1 + 0.2 * xx)
    x[..., 1] = (xx ** 2 + yy ** 2 < 0.05)
    x = cn.bf16_round(x)
    tval = np.sqrt(xx ** 2 + yy ** 2)[None].repeat(B, 0).astype(np.float32) / 2
    tctrl = ((np.arctan2(yy, xx) + np.pi) / (2 * np.pi) * 32).astype(np.uint8)[None].repeat(B, 0) % 32
    free = np.ones((B, H, W), np.uint8)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    xd = dev(cn.bf16_bits(x).view(np.int16))
    args = (dev(tval), dev(tctrl), dev(free), int(free.sum()))
    first = net.train_step(xd, *args, lr=2e-3, w_value=1.0, w_ctrl=0.1)
    for _ in range(300):
        last = net.train_step(xd, *args, lr=2e-3, w_value=1.0, w_ctrl=0.1)
    assert last[0] < 0.2 * first[0] and last[1] < 0.8 * first[1], (first, last)
    net.close()
