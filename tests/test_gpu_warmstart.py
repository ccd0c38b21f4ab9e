"""Warm-start plumbing: batch <-> field bridges, data preparation kernels, and
a small end-to-end run (generate, train, relax with and without the network).
"""
import numpy as np
import pytest

from gen.images import two_phase_materials, warmstart_specimens

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04565_gb300 import batch, build, lsm, nn, warmstart
    build.build()
    nn.lib()
    return torch, batch, lsm, nn, warmstart


def test_fields_and_add_displacements(env):
    torch, batch, lsm, nn, ws = env
    imgs = warmstart_specimens(range(3), side=32)
    k, e, m = two_phase_materials()
    bt = batch.Batch(imgs, k, e, m, precision="exact64", **ws.RELAX)
    bt.apply_strain(0.01)
    bt.step(30)
    f = ws.Fields(3, 32, 32)
    f.read(bt, with_phase=True)
    torch.cuda.synchronize()
    X = np.stack(np.meshgrid(np.arange(32.0), np.arange(32.0), indexing="xy")).reshape(2, -1)
    for q in range(3):
        x, _ = bt.state(q)
        u = f.u[q].cpu().numpy().reshape(2, -1)
        assert np.allclose(u, (x - X).astype(np.float32), rtol=0, atol=1e-6)
        assert np.array_equal(f.phase[q].cpu().numpy(), imgs[q])
    rng = np.random.default_rng(0)
    du = (1e-3 * rng.standard_normal((3, 2, 32, 32))).astype(np.float32)
    before = [bt.state(q)[0] for q in range(3)]
    tdu = torch.from_numpy(du).cuda()
    nn.check(nn.lib().lsm_batch_add_displacements(bt.h, nn.ptr(tdu), 32, 32), bt.h, batch=True)
    torch.cuda.synchronize()
    for q in range(3):
        x, _ = bt.state(q)
        d = du[q].reshape(2, -1).astype(np.float64)
        grip = (np.arange(32 * 32) % 32 == 0) | (np.arange(32 * 32) % 32 == 31)
        d[0, grip] = 0.0  # roller grips: x prescribed
        assert np.array_equal(x, before[q] + d)


def test_prepare_kernels(env):
    torch, batch, lsm, nn, ws = env
    S, H, W = 2, 16, 24
    rng = np.random.default_rng(1)
    phase = rng.integers(1, 3, size=(S, H, W)).astype(np.uint8)
    u = rng.standard_normal((S, 2, H, W)).astype(np.float32) * 1e-2
    eps = np.array([0.01, 0.02], np.float32)
    tph, tu, te = (torch.from_numpy(a).cuda() for a in (phase, u, eps))
    xin = torch.zeros((S, H, W, 32), dtype=torch.bfloat16, device="cuda")
    nn.check(nn.lib().lsm_unet_prepare_input(nn.ptr(tph), nn.ptr(tu), nn.ptr(te), 1e-3, S, H, W, 1.0, nn.ptr(xin),
                                             None))
    torch.cuda.synchronize()
    got = xin.float().cpu().numpy()
    Xx = np.arange(W)[None, None, :] - 0.5 * (W - 1)
    Yy = np.arange(H)[None, :, None] - 0.5 * (H - 1)
    us = eps[:, None, None] * 0.5 * W
    ref = np.zeros((S, H, W, 32), np.float32)
    ref[..., 0] = phase - 1.5
    ref[..., 1] = (u[:, 0] - eps[:, None, None] * Xx) / us
    ref[..., 2] = u[:, 1] / us
    ref[..., 3] = 1.0
    ref[..., 4] = eps[:, None, None] / 0.1
    ref[..., 5] = np.broadcast_to(Xx / (0.5 * W), (S, H, W))
    ref[..., 6] = np.broadcast_to(Yy / (0.5 * H), (S, H, W))
    assert np.allclose(got, ref, rtol=2 ** -7, atol=1e-6)
    # target and its inverse map
    u2 = u + 1e-3 * rng.standard_normal(u.shape).astype(np.float32)
    tu2 = torch.from_numpy(u2).cuda()
    tgt = torch.zeros((S, H, W, 2), dtype=torch.float32, device="cuda")
    nn.check(nn.lib().lsm_unet_prepare_target(nn.ptr(tu), nn.ptr(tu2), 1e-3, S, H, W, 1.0, nn.ptr(tgt), None))
    du = torch.zeros((S, 2, H, W), dtype=torch.float32, device="cuda")
    nn.check(nn.lib().lsm_unet_prediction_to_displacement(nn.ptr(tgt), 1e-3, S, H, W, 1.0, nn.ptr(du), None))
    torch.cuda.synchronize()
    assert np.allclose(du.cpu().numpy(), u2 - u, rtol=1e-5, atol=1e-9)


def test_warm_start_end_to_end_small(env):
    """Generate data on small specimens, train briefly, and relax the same
    increments with and without the prediction: both reach the tolerance and
    land on the same equilibrium (to the tolerance's resolution)."""
    torch, batch, lsm, nn, ws = env
    k, e, m = two_phase_materials()
    imgs = warmstart_specimens(range(8), side=32)
    data = ws.generate(imgs, k, e, m, increments=4, tol=1e-7)
    assert data["U"].shape[0] == 32
    net, info = ws.train(data, steps=150, batch=8, lr=2e-3)
    first, last = info["loss_history"][0][1], info["loss_history"][-1][1]
    assert last < first
    res = ws.compare(imgs[:4], k, e, m, net, first_inc=2, increments=1, tol=1e-8, precision="df64")
    for arm in ("plain", "batched", "warm"):
        assert res[arm]["seconds_per_increment"] > 0
    assert res["batched"]["converged"] == res["warm"]["converged"] == 4


def test_warm_start_reduces_relaxation_steps(env):
    """What the trained network gains over the method without it. The network
    is trained on increments the method itself relaxed (64 specimens of
    64 x 64, their pre-fracture increments, 6,000 Adam steps) and predicts
    each increment of 8 held-out specimens: with the prediction added after
    the load step, the batched relaxation needs at least 5% fewer steps to
    the same force residual (1e-8, the warm-start configuration's tolerance),
    summed over the held-out specimens' increments (all before fracture);
    both arms end in the same equilibrium, up to a rigid translation along
    y (roller grips prescribe x only, so the relaxation never removes a
    uniform y shift in the prediction). (Measured on a GB300: 7.8% fewer
    steps at a held-out prediction error of 0.15; the exact relaxed field as
    the prediction, stored in FP32 like the network's output, gives 4.8x
    fewer. The relaxation is underdamped, every mode decays at the same rate
    gamma / 2, so steps fall with the logarithm of the starting error.)"""
    torch, batch, lsm, nn, ws = env
    k, e, m = two_phase_materials()
    data = ws.generate(warmstart_specimens(range(64), side=64), k, e, m, increments=8, tol=1e-7,
                       precision="df64", pre_fracture=True)
    assert data["U"].shape[0] >= 400  # specimens x increments before any break
    net, _ = ws.train(data, steps=6000, batch=8, lr=1e-3)
    held = warmstart_specimens(range(3000, 3008), side=64)
    res = ws.steps_to_tolerance(held, k, e, m, net, increments=6, tol=1e-8, check_every=10)
    b, w = res["batched"], res["warm"]
    assert all(all(c) for c in b["converged"]) and all(all(c) for c in w["converged"])
    assert all(fb < 0 for fb in b["first_break"]) and all(fb < 0 for fb in w["first_break"])
    sb = sum(map(sum, b["steps"]))
    sw = sum(map(sum, w["steps"]))
    per_inc = [(sum(x), sum(y)) for x, y in zip(b["steps"], w["steps"])]
    print("relaxation steps to 1e-8, 8 held-out specimens x 6 increments: batched %d, warm start %d "
          "(%.3f); per increment %s" % (sb, sw, sw / sb, per_inc))
    assert sw <= 0.95 * sb
    for q in range(len(held)):
        d = w["x"][q] - b["x"][q]
        d[1] -= d[1].mean()  # the rigid y translation the grips leave free
        assert np.abs(d).max() <= 1e-4
        assert w["last"][q]["sigma_vir"] == pytest.approx(b["last"][q]["sigma_vir"], rel=1e-4)
        assert w["last"][q]["residual"] <= 1e-8 and b["last"][q]["residual"] <= 1e-8
