"""FP64 CPU reference of the warm-start U-Net -- TEST INFRASTRUCTURE ONLY.

Plain numpy forward pass and hand-written backward pass of the network the
CUDA library trains (see include/lsm_nn.h): 14 3x3 convolutions with bias and
ReLU in a 4-level U-Net (32/64/128/256 channels, 2x2 max pooling with the
first maximum of each window, nearest x2 upsampling, skip concatenation
[upsampled | encoder]), a 1x1 head to 2 channels, mean squared error.

Parameter layout (flat FP32/FP64 vector, identical to the library's): for
each conv q, W[q] as [Cout][3][3][Cin] then bias[Cout]; then the head's
W [2][32] and bias [2].

With rounding=True the reference rounds to BF16 at exactly the points where
the GPU stores BF16 (conv outputs, dense activation gradients), so that GPU
and reference differ only by FP32-vs-FP64 accumulation; with rounding=False
it is plain FP64 (used for the finite-difference pin).
"""
from __future__ import annotations

import numpy as np

CONVS = [(32, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (128, 256),
         (256, 256), (384, 128), (128, 128), (192, 64), (64, 64), (96, 32), (32, 32)]


def layout():
    """(offsets of W, offsets of b) per conv, head W, head b, total count."""
    off, wo, bo = 0, [], []
    for cin, cout in CONVS:
        wo.append(off)
        off += cout * 9 * cin
        bo.append(off)
        off += cout
    hw = off
    off += 64
    hb = off
    off += 2
    return wo, bo, hw, hb, off


def bf16(x):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    x32 = np.ascontiguousarray(x, dtype=np.float32)
    b = x32.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _shift(x, dy, dx):
    """y[b, i, j] = x[b, i + dy, j + dx] (zero outside)."""
    B, H, W, C = x.shape
    y = np.zeros_like(x)
    ys, ye = max(0, -dy), min(H, H - dy)
    xs, xe = max(0, -dx), min(W, W - dx)
    y[:, ys:ye, xs:xe] = x[:, ys + dy:ye + dy, xs + dx:xe + dx]
    return y


def conv(x, W, b):
    """3x3 convolution, zero padding 1: out = b + sum_taps shift(x) @ W[:, tap].T"""
    out = np.zeros(x.shape[:3] + (W.shape[0],))
    for ky in range(3):
        for kx in range(3):
            out += np.tensordot(_shift(x, ky - 1, kx - 1), W[:, ky, kx, :], axes=([3], [1]))
    return out + b


def conv_bwd(x, W, g):
    """Gradients of conv w.r.t. W, b and x for the output gradient g."""
    dW = np.zeros_like(W)
    dx = np.zeros_like(x)
    for ky in range(3):
        for kx in range(3):
            xs = _shift(x, ky - 1, kx - 1)
            dW[:, ky, kx, :] = np.tensordot(g, xs, axes=([0, 1, 2], [0, 1, 2]))
            dx += _shift(np.tensordot(g, W[:, ky, kx, :], axes=([3], [0])), 1 - ky, 1 - kx)
    return dW, g.sum(axis=(0, 1, 2)), dx


def pool(x):
    B, H, W, C = x.shape
    v = x.reshape(B, H // 2, 2, W // 2, 2, C)
    return v.max(axis=(2, 4))


def pool_bwd(x, g):
    """Gradient of the 2x2 max pool routed to the first maximum of each window
    (window order (0,0), (0,1), (1,0), (1,1))."""
    B, H, W, C = x.shape
    v = x.reshape(B, H // 2, 2, W // 2, 2, C).transpose(0, 1, 3, 2, 4, 5).reshape(B, H // 2, W // 2, 4, C)
    arg = v.argmax(axis=3)  # first maximum
    out = np.zeros((B, H // 2, W // 2, 4, C))
    np.put_along_axis(out, arg[:, :, :, None, :], g[:, :, :, None, :], axis=3)
    return out.reshape(B, H // 2, W // 2, 2, 2, C).transpose(0, 1, 3, 2, 4, 5).reshape(B, H, W, C)


def up(x):
    return x.repeat(2, axis=1).repeat(2, axis=2)


def up_bwd(g):
    B, H, W, C = g.shape
    return g.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def unpack(params):
    wo, bo, hw, hb, n = layout()
    assert params.size == n
    Ws, bs = [], []
    for q, (cin, cout) in enumerate(CONVS):
        Ws.append(params[wo[q]:wo[q] + cout * 9 * cin].reshape(cout, 3, 3, cin))
        bs.append(params[bo[q]:bo[q] + cout])
    return Ws, bs, params[hw:hw + 64].reshape(2, 32), params[hb:hb + 2]


def forward(params, x, rounding=True):
    """Returns (output [B, H, W, 2], cache)."""
    R = bf16 if rounding else (lambda a: a)
    Ws, bs, Wh, bh = unpack(np.asarray(params, dtype=np.float64))
    if rounding:
        Ws = [bf16(w) for w in Ws]
    c = {"x": x}

    def cv(q, inp):
        return R(np.maximum(conv(inp, Ws[q], bs[q]), 0.0))

    c["e1a"] = cv(0, x)
    c["e1"] = cv(1, c["e1a"])
    c["p1"] = pool(c["e1"])
    c["e2a"] = cv(2, c["p1"])
    c["e2"] = cv(3, c["e2a"])
    c["p2"] = pool(c["e2"])
    c["e3a"] = cv(4, c["p2"])
    c["e3"] = cv(5, c["e3a"])
    c["p3"] = pool(c["e3"])
    c["e4a"] = cv(6, c["p3"])
    c["e4"] = cv(7, c["e4a"])
    c["d3c"] = np.concatenate([up(c["e4"]), c["e3"]], axis=3)
    c["d3a"] = cv(8, c["d3c"])
    c["d3"] = cv(9, c["d3a"])
    c["d2c"] = np.concatenate([up(c["d3"]), c["e2"]], axis=3)
    c["d2a"] = cv(10, c["d2c"])
    c["d2"] = cv(11, c["d2a"])
    c["d1c"] = np.concatenate([up(c["d2"]), c["e1"]], axis=3)
    c["d1a"] = cv(12, c["d1c"])
    c["d1"] = cv(13, c["d1a"])
    out = np.tensordot(c["d1"], Wh, axes=([3], [1])) + bh
    c.update(Ws=Ws, Wh=Wh)
    return out, c


def loss_and_grad(params, x, target, rounding=True):
    """Mean squared error and its gradient w.r.t. the flat parameter vector."""
    R = bf16 if rounding else (lambda a: a)
    out, c = forward(params, x, rounding)
    n = out.size
    loss = float(((out - target) ** 2).sum() / n)
    gout = 2.0 * (out - target) / n
    wo, bo, hw, hb, N = layout()
    grad = np.zeros(N)
    Ws, Wh = c["Ws"], c["Wh"]
    grad[hw:hw + 64] = np.tensordot(gout, c["d1"], axes=([0, 1, 2], [0, 1, 2])).reshape(-1)
    grad[hb:hb + 2] = gout.sum(axis=(0, 1, 2))

    def mask(g, act):
        return np.where(act > 0, g, 0.0)

    def cb(q, g, inp, want_dx=True):
        dW, db, dx = conv_bwd(inp, Ws[q], g)
        cin, cout = CONVS[q]
        grad[wo[q]:wo[q] + cout * 9 * cin] = dW.reshape(-1)
        grad[bo[q]:bo[q] + cout] = db
        return R(dx) if want_dx else None

    g = R(mask(np.tensordot(gout, Wh, axes=([3], [0])), c["d1"]))
    g = mask(cb(13, g, c["d1a"]), c["d1a"])
    gd1c = cb(12, g, c["d1c"])
    g = mask(R(up_bwd(gd1c[..., :64])), c["d2"])
    g = mask(cb(11, g, c["d2a"]), c["d2a"])
    gd2c = cb(10, g, c["d2c"])
    g = mask(R(up_bwd(gd2c[..., :128])), c["d3"])
    g = mask(cb(9, g, c["d3a"]), c["d3a"])
    gd3c = cb(8, g, c["d3c"])
    g = mask(R(up_bwd(gd3c[..., :256])), c["e4"])
    g = mask(cb(7, g, c["e4a"]), c["e4a"])
    g = cb(6, g, c["p3"])
    g = mask(R(pool_bwd(c["e3"], g) + gd3c[..., 256:]), c["e3"])
    g = mask(cb(5, g, c["e3a"]), c["e3a"])
    g = cb(4, g, c["p2"])
    g = mask(R(pool_bwd(c["e2"], g) + gd2c[..., 128:]), c["e2"])
    g = mask(cb(3, g, c["e2a"]), c["e2a"])
    g = cb(2, g, c["p1"])
    g = mask(R(pool_bwd(c["e1"], g) + gd1c[..., 64:]), c["e1"])
    g = mask(cb(1, g, c["e1a"]), c["e1a"])
    cb(0, g, c["x"], want_dx=False)
    return loss, grad, out
