"""FP64 CPU reference of the learned warm start's layers -- test infrastructure
only (imported by tests, never by the product path).

The network is not in the paper: it stands in for the initial value of the
coarse solve (Section 4.3, "Initialization").  Each function here is the
textbook definition of its layer written out in float64 numpy, with no
blocking or reordering:

* ``conv3x3``: y[b, i, j, o] = sum_{t, c} w[o, t, c] x[b, i + d dy_t, j + d dx_t, c]
  (+ bias, optional ReLU), taps t = 3 (dy + 1) + (dx + 1), dilation d, zero outside
  the image;
* ``conv3x3_dgrad``: the adjoint of conv3x3 in x (optionally times a ReLU mask);
* ``conv3x3_wgrad``: the gradient of sum(dy * conv3x3(x, w)) in w and the bias;
* ``loss_and_grad``: squared value error plus softmax cross-entropy of the
  control logits over the counted pixels, and its gradient in the outputs.

Images are NHWC arrays; w has shape (cout, 9, cin).
"""
from __future__ import annotations

import numpy as np

TAPS = [(t // 3 - 1, t % 3 - 1) for t in range(9)]


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (round to nearest, ties to even) and
    return them as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def bf16_bits(a: np.ndarray) -> np.ndarray:
    """The bfloat16 bit patterns (uint16) of bf16_round(a)."""
    r = bf16_round(a).astype(np.float32)
    return (r.view(np.uint32) >> 16).astype(np.uint16)


def _shifted(x: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """s[b, i, j] = x[b, i + dy, j + dx], zero outside the image."""
    B, H, W = x.shape[:3]
    s = np.zeros_like(x)
    i0, i1 = max(0, -dy), min(H, H - dy)
    j0, j1 = max(0, -dx), min(W, W - dx)
    if i1 > i0 and j1 > j0:          # a shift past the image reads only zeros
        s[:, i0:i1, j0:j1] = x[:, i0 + dy:i1 + dy, j0 + dx:j1 + dx]
    return s


def conv3x3(x, w, b=None, relu=False, dil=1):
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    y = np.zeros(x.shape[:3] + (w.shape[0],))
    for t, (dy, dx) in enumerate(TAPS):
        y += np.einsum("bijc,oc->bijo", _shifted(x, dil * dy, dil * dx), w[:, t, :])
    if b is not None:
        y += np.asarray(b, dtype=np.float64)
    return np.maximum(y, 0.0) if relu else y


def conv3x3_dgrad(dy, w, mask=None, dil=1):
    """dx[b, i, j, c] = sum_{t, o} w[o, t, c] dy[b, i - d dy_t, j - d dx_t, o]."""
    dy = np.asarray(dy, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    dx = np.zeros(dy.shape[:3] + (w.shape[2],))
    for t, (oy, ox) in enumerate(TAPS):
        dx += np.einsum("bijo,oc->bijc", _shifted(dy, -dil * oy, -dil * ox), w[:, t, :])
    if mask is not None:
        dx = dx * (np.asarray(mask) > 0)
    return dx


def conv3x3_wgrad(x, dy, dil=1):
    """dw[o, t, c] = sum_{b, i, j} dy[b, i, j, o] x[b, i + d dy_t, j + d dx_t, c];
    db[o] = sum dy[..., o]."""
    x = np.asarray(x, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    dw = np.zeros((dy.shape[3], 9, x.shape[3]))
    for t, (oy, ox) in enumerate(TAPS):
        dw[:, t, :] = np.einsum("bijo,bijc->oc", dy, _shifted(x, dil * oy, dil * ox))
    return dw, dy.sum(axis=(0, 1, 2))


def loss_and_grad(out, tval, tctrl, free, wv, wc):
    """out[..., 0] is the value, out[..., 1:1+n] the control logits.  Over the
    counted pixels: Lv = mean (o0 - tval)^2, Lc = mean (log sum exp(o) - o[tctrl]);
    returns (Lv, Lc, d(wv Lv + wc Lc)/d out)."""
    out = np.asarray(out, dtype=np.float64)
    m = np.asarray(free).astype(bool)
    nf = max(1, int(m.sum()))
    g = np.zeros_like(out)
    d = out[..., 0] - tval
    lv = float((d[m] ** 2).sum() / nf)
    g[..., 0] = np.where(m, 2.0 * d * wv / nf, 0.0)
    logits = out[..., 1:33]
    mx = logits.max(axis=-1, keepdims=True)
    e = np.exp(logits - mx)
    p = e / e.sum(axis=-1, keepdims=True)
    idx = np.asarray(tctrl).astype(np.int64)
    picked = np.take_along_axis(logits, idx[..., None], axis=-1)[..., 0]
    lse = np.log(e.sum(axis=-1)) + mx[..., 0]
    lc = float((lse - picked)[m].sum() / nf)
    onehot = np.zeros_like(p)
    np.put_along_axis(onehot, idx[..., None], 1.0, axis=-1)
    g[..., 1:33] = np.where(m[..., None], (p - onehot) * wc / nf, 0.0)
    return lv, lc, g
