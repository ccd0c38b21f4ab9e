"""Pins of the FP64 U-Net reference (oracle/unet_ref.py) on the CPU.

Its hand-written backward pass must agree with central finite differences of
its own forward loss (plain FP64, no BF16 rounding); its convolution must
agree with a direct per-pixel sum; its pooling/upsampling adjoints must
satisfy <A x, y> = <x, A^T y>.
"""
import numpy as np
import pytest

from oracle import unet_ref as R


def _rand_params(rng, scale=0.3):
    *_, n = R.layout()
    return scale * rng.standard_normal(n)


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 6, 3))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    out = R.conv(x, W, b)
    for (bb, i, j, o) in [(0, 0, 0, 0), (1, 4, 5, 3), (0, 2, 3, 1), (1, 0, 5, 2)]:
        s = b[o]
        for ky in range(3):
            for kx in range(3):
                ii, jj = i + ky - 1, j + kx - 1
                if 0 <= ii < 5 and 0 <= jj < 6:
                    s += W[o, ky, kx] @ x[bb, ii, jj]
        assert out[bb, i, j, o] == pytest.approx(s, rel=1e-12)


def test_pool_and_up_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 8, 6, 3))
    g = rng.standard_normal((2, 4, 3, 3))
    # pool_bwd is the adjoint of the (fixed-argmax) selection
    lhs = (R.pool(x) * g).sum()
    rhs = (x * R.pool_bwd(x, g)).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)
    y = rng.standard_normal((2, 8, 6, 3))
    assert (R.up(g) * y).sum() == pytest.approx((g * R.up_bwd(y)).sum(), rel=1e-12)
    # ties go to the first maximum of the window
    t = np.zeros((1, 2, 2, 1))
    gb = R.pool_bwd(t, np.ones((1, 1, 1, 1)))
    assert gb[0, 0, 0, 0] == 1.0 and gb.sum() == 1.0


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    params = _rand_params(rng)
    x = np.zeros((1, 8, 8, 32))
    x[..., :4] = rng.standard_normal((1, 8, 8, 4))
    target = rng.standard_normal((1, 8, 8, 2))
    loss, grad, _ = R.loss_and_grad(params, x, target, rounding=False)
    wo, bo, hw, hb, n = R.layout()
    picks = [wo[0] + 3, wo[0] + 2 * 9 * 32 + 1, bo[1], wo[5] + 77, bo[7] + 2, wo[8] + 1000, wo[12] + 5,
             wo[13] + 11, bo[13], hw + 7, hb + 1, wo[6] + 300, wo[10] + 4000]
    h = 1e-6
    for i in picks:
        p1 = params.copy(); p1[i] += h
        p2 = params.copy(); p2[i] -= h
        fd = (R.loss_and_grad(p1, x, target, rounding=False)[0] -
              R.loss_and_grad(p2, x, target, rounding=False)[0]) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=2e-5, abs=1e-9 * max(1.0, abs(loss))), i


def test_bf16_rounding_is_round_to_nearest_even():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 1e-3])
    r = R.bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -6 and r[3] == -2.5
    assert abs(r[4] - 1e-3) <= 2 ** -8 * 1e-3
