"""U-Net tensor-core kernels vs the FP64 CPU reference (oracle/unet_ref.py).

The reference rounds to BF16 where the GPU stores BF16, so the remaining
differences come from FP32 (GPU) vs FP64 (reference) accumulation and from
the occasional BF16 rounding that lands on the other side of a tie."""
import numpy as np
import pytest

from oracle import unet_ref as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04565_gb300 import build, nn
    build.build()
    nn.lib()
    return torch, nn


def _bf(torch, a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("cin,cout,taps,relu,B,H,W", [(64, 64, 9, 1, 2, 8, 12), (96, 32, 9, 0, 2, 8, 12),
                                                       (32, 128, 1, 1, 2, 8, 12), (384, 128, 9, 1, 2, 8, 12),
                                                       (32, 256, 9, 1, 2, 16, 32), (192, 384, 9, 0, 1, 5, 70),
                                                       (64, 96, 9, 1, 3, 33, 130), (128, 64, 1, 0, 2, 4, 3),
                                                       (32, 64, 9, 1, 2, 20, 8), (64, 32, 9, 0, 1, 17, 5),
                                                       (64, 128, 9, 1, 1, 153, 100), (32, 64, 1, 0, 2, 160, 64)])
def test_conv_forward_matches_reference(env, cin, cout, taps, relu, B, H, W):
    """The tensor-core forward convolution against the reference, on channel
    slices of wider tensors: patches of 128 pixels (whole, ragged, narrower
    than the image), 32- and 64-channel K chunks, output tiles of 32 to 256
    channels, one or several; the variant with resident weights and halo
    copies (3x3, up to 64 output channels a tile, patches 16 or 8 pixels wide)
    and the one streaming weights per tap (1x1, wider output tiles), with two
    patches per work item once the patches outnumber the SMs (153 patches:
    an odd count, the last item's second patch read as zeros and not
    stored)."""
    torch, nn = env
    rng = np.random.default_rng(cin + cout + W)
    cs_in, c0_in, cs_out, c0_out = cin + 32, 32, cout + 64, 64  # channel slices of wider tensors
    x = R.bf16(rng.standard_normal((B, H, W, cs_in)))
    Wt = R.bf16(0.2 * rng.standard_normal((cout, taps, cin)))
    b = rng.standard_normal(cout).astype(np.float32).astype(np.float64)
    out = torch.zeros((B, H, W, cs_out), dtype=torch.bfloat16, device="cuda")
    tb = torch.from_numpy(b.astype(np.float32)).cuda()
    tx, tw = _bf(torch, x), _bf(torch, Wt)  # keep the buffers alive until the kernel has run
    nn.check(nn.lib().lsm_nn_conv_forward(nn.ptr(tx), cs_in, c0_in, cin, nn.ptr(tw), nn.ptr(tb),
                                          nn.ptr(out), cs_out, c0_out, cout, B, H, W, taps, relu, None))
    torch.cuda.synchronize()
    got = out.float().cpu().numpy().astype(np.float64)
    xi = x[..., c0_in:c0_in + cin]
    if taps == 9:
        ref = R.conv(xi, Wt.reshape(cout, 3, 3, cin), b)
    else:
        ref = np.tensordot(xi, Wt[:, 0, :], axes=([3], [1])) + b
    if relu:
        ref = np.maximum(ref, 0.0)
    ref = R.bf16(ref)
    g = got[..., c0_out:c0_out + cout]
    assert np.all(got[..., :c0_out] == 0.0)  # nothing written outside the slice
    err = np.abs(g - ref)
    assert np.all(err <= 2 ** -7 * np.abs(ref) + 1e-6 * np.abs(ref).max())


def test_conv_wait_timeout_is_reported_and_recovers(env):
    """Fault injection without a GPU fault: with a wait limit of 0 polls the
    tensor-core convolution's first bounded mbarrier wait gives up at once;
    the CTA drains the MMAs it issued, frees its tensor memory and the call
    returns LSM_ETIMEOUT. At the default limit the next call on the same
    buffers computes the right result."""
    torch, nn = env
    from paper_2201_04565_gb300 import lsm
    rng = np.random.default_rng(3)
    B, H, W, cin, cout = 2, 16, 16, 64, 64
    x = R.bf16(rng.standard_normal((B, H, W, cin)))
    Wt = R.bf16(0.2 * rng.standard_normal((cout, 9, cin)))
    b = rng.standard_normal(cout).astype(np.float32).astype(np.float64)
    out = torch.zeros((B, H, W, cout), dtype=torch.bfloat16, device="cuda")
    tb = torch.from_numpy(b.astype(np.float32)).cuda()
    tx, tw = _bf(torch, x), _bf(torch, Wt)
    L = nn.lib()

    def run():
        return L.lsm_nn_conv_forward(nn.ptr(tx), cin, 0, cin, nn.ptr(tw), nn.ptr(tb), nn.ptr(out), cout, 0,
                                     cout, B, H, W, 9, 0, None)

    nn.check(L.lsm_nn_set_wait_limit(0, None))
    try:
        assert run() == lsm.LSM_ETIMEOUT
    finally:
        nn.check(L.lsm_nn_set_wait_limit(-1, None))
    nn.check(run())
    torch.cuda.synchronize()
    got = out.float().cpu().numpy().astype(np.float64)
    ref = R.bf16(R.conv(x, Wt.reshape(cout, 3, 3, cin), b))
    assert np.all(np.abs(got - ref) <= 2 ** -7 * np.abs(ref) + 1e-6 * np.abs(ref).max())


@pytest.mark.parametrize("cin,cout,taps,B,H,W", [(64, 64, 9, 2, 9, 14), (32, 256, 9, 2, 9, 14),
                                                  (96, 32, 1, 2, 9, 14), (128, 64, 9, 2, 40, 37),
                                                  (256, 160, 9, 1, 20, 21), (32, 32, 9, 2, 32, 64),
                                                  (192, 128, 9, 1, 16, 130)])
def test_conv_wgrad_matches_reference(env, cin, cout, taps, B, H, W):
    """The tensor-core weight gradient (tiles of 128 (tap, input channel)
    rows, the last one partly filled, x 32 to 256 output channels; patches of
    64 pixels, whole and ragged; one or several pixel splits) against the
    reference."""
    torch, nn = env
    rng = np.random.default_rng(7 + cin)
    x = R.bf16(rng.standard_normal((B, H, W, cin)))
    g = R.bf16(rng.standard_normal((B, H, W, cout)))
    dW = torch.zeros(cout * taps * cin, dtype=torch.float32, device="cuda")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda")
    ws = torch.zeros(1 << 20, dtype=torch.float32, device="cuda")
    tg, tx = _bf(torch, g), _bf(torch, x)
    nn.check(nn.lib().lsm_nn_conv_wgrad(nn.ptr(tg), cout, nn.ptr(tx), cin, 0, cin, B, H, W, taps,
                                        nn.ptr(dW), nn.ptr(db), nn.ptr(ws), ws.numel(), None))
    torch.cuda.synchronize()
    if taps == 9:
        rdW, rdb, _ = R.conv_bwd(x, np.zeros((cout, 3, 3, cin)), g)
        rdW = rdW.reshape(cout, 9, cin)
    else:
        rdW = np.tensordot(g, x, axes=([0, 1, 2], [0, 1, 2]))[:, None, :]
        rdb = g.sum(axis=(0, 1, 2))
    gdW = dW.cpu().numpy().reshape(cout, taps, cin)
    assert np.abs(gdW - rdW).max() <= 1e-4 * np.abs(rdW).max()
    assert np.abs(db.cpu().numpy() - rdb).max() <= 1e-4 * np.abs(rdb).max()


def _net_inputs(rng, B, H, W):
    x = np.zeros((B, H, W, 32))
    x[..., :4] = rng.standard_normal((B, H, W, 4))
    return R.bf16(x), rng.standard_normal((B, H, W, 2)).astype(np.float32).astype(np.float64)


def test_unet_loss_and_gradients_match_reference(env):
    """Loss and every parameter block's gradient vs the reference. BF16
    storage of activations and gradients (and the ReLU masks it can flip) make
    even the BF16-emulating reference differ from plain FP64 by several
    percent; the GPU must stay within that noise floor of the emulation."""
    torch, nn = env
    B, H, W = 2, 32, 32
    net = nn.UNet(H, W, B, seed=3)
    params = net.get_params().astype(np.float64)
    rng = np.random.default_rng(4)
    x, t = _net_inputs(rng, B, H, W)
    tx = _bf(torch, x)
    tt = torch.from_numpy(t.astype(np.float32)).cuda()
    out = torch.zeros((B, H, W, 2), dtype=torch.float32, device="cuda")
    net.forward(tx, out, B)
    loss, grad = net.gradients(tx, tt, B)
    rloss, rgrad, rout = R.loss_and_grad(params, x, t, rounding=True)
    _, rgrad64, _ = R.loss_and_grad(params, x, t, rounding=False)
    got = out.cpu().numpy()
    assert np.abs(got - rout).max() <= 2e-2 * np.abs(rout).max()
    assert loss == pytest.approx(rloss, rel=1e-2)
    wo, bo, hw, hb, n = R.layout()
    blocks = [(wo[q], bo[q]) for q in range(14)] + [(bo[q], bo[q] + R.CONVS[q][1]) for q in range(14)]
    blocks += [(hw, hw + 64), (hb, hb + 2)]
    worst = 0.0
    for a, b in blocks:
        nr = max(np.linalg.norm(rgrad[a:b]), 1e-30)
        e = np.linalg.norm(grad[a:b] - rgrad[a:b]) / nr
        noise = np.linalg.norm(rgrad64[a:b] - rgrad[a:b]) / nr  # BF16 effect in the reference itself
        # rounding noise of the same order as the emulation's own; a wrong
        # index or sign anywhere gives O(1) errors instead
        assert e <= max(1.25 * noise, 2e-2), (a, b, e, noise)
        worst = max(worst, e)
    print("worst normwise gradient error per block: %.3e" % worst)
    assert worst <= 0.15


def test_training_reduces_loss(env):
    torch, nn = env
    B, H, W = 4, 32, 32
    net = nn.UNet(H, W, B, seed=5)
    rng = np.random.default_rng(6)
    x = np.zeros((B, H, W, 32))
    x[..., :4] = rng.standard_normal((B, H, W, 4))
    # a smooth target that depends on the input: blurred channel sums
    t = np.stack([x[..., 0] + 0.5 * x[..., 1], x[..., 2] - x[..., 3]], axis=-1)
    tx = _bf(torch, R.bf16(x))
    tt = torch.from_numpy(t.astype(np.float32)).cuda()
    first = net.train_step(tx, tt, B, 2e-3)
    for _ in range(300):
        last = net.train_step(tx, tt, B, 2e-3, want_loss=False)
    last = net.train_step(tx, tt, B, 2e-3)
    assert last < 0.1 * first, (first, last)
