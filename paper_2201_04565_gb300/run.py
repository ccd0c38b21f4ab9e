"""Command-line runs of the lattice-spring path on seeded synthetic specimens.

  python -m paper_2201_04565_gb300.run single --side 2048 --precision df64 --increments 3
  python -m paper_2201_04565_gb300.run foam --side 96 --precision df64 --increments 3
  python -m paper_2201_04565_gb300.run batch --count 64 --precision df64 --increments 3
  python -m paper_2201_04565_gb300.run unet --side 256 --batch 8 --iters 3
  python -m paper_2201_04565_gb300.run conv --side 256 --batch 8 --iters 20

single: a 2D two-phase inclusion composite (fused tile kernel, or the
spring-list kernels with --path 1); foam: a 3D one-phase foam under
compression (voxel tile kernel in df64 / f32, spring-list kernels in the FP64
modes or with --path 1); batch: uneven 2D specimens (sides 32 to
--max-side) in one batched context; unet: training iterations of the
warm-start network on random inputs; conv: each of the network's 14
convolution shapes on its own (forward, and weight gradient), timed with CUDA
events on random BF16 operands, in TFLOP/s. Each tension case runs a displacement-controlled
tension (or compression) test of --increments load increments of --steps time
steps and prints a one-line JSON summary (last stress sample, broken springs,
kernel launches).
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import sys
import time


def _single(a):
    from gen.images import inclusion_image, two_phase_materials

    from . import lsm
    img = inclusion_image(a.side, a.side, 10.0, 60.0, 0.30, a.seed)
    k, e, m = two_phase_materials()
    sp = lsm.Specimen.from_image(img, k, e, m, dt=0.01, damping=0.1, precision=a.precision, path=a.path,
                                 lattice=a.lattice)
    t0 = time.perf_counter()
    if a.rate:  # one increment, then the grips at a constant strain rate (eps_inc per `steps` steps)
        sp.apply_strain(a.eps_inc)
        sp.set_strain_rate(a.eps_inc / (a.steps * 0.01))
    for i in range(1, a.increments + 1):
        if not a.rate:
            sp.apply_strain(i * a.eps_inc)
        sp.step(a.steps)
    sp.synchronize()
    dt = time.perf_counter() - t0
    s = sp.samples()[-1]
    out = {"case": "single", "side": a.side, "particles": sp.n, "springs": sp.m, "seconds": dt,
           "last_sample": s, "kernel_launches": sp.counters()[2]}
    sp.close()
    return out


def _foam(a):
    from gen.images import foam_volume, one_phase_materials

    from . import lsm
    img = foam_volume(a.side, 3.0, 0.40, seed=a.seed)
    k, e, m = one_phase_materials(1.0, 0.04)
    sp = lsm.Specimen.from_image(img, k, e, m, dt=0.01, damping=0.1, precision=a.precision, grip_mode=1,
                                 path=a.path)
    t0 = time.perf_counter()
    for i in range(1, a.increments + 1):
        sp.apply_strain(-i * a.eps_inc)
        sp.step(a.steps)
    sp.synchronize()
    dt = time.perf_counter() - t0
    s = sp.samples()[-1]
    out = {"case": "foam", "side": a.side, "particles": sp.n, "springs": sp.m, "seconds": dt,
           "last_sample": s, "kernel_launches": sp.counters()[2]}
    sp.close()
    return out


def _batch(a):
    from gen.images import batch_specimens, two_phase_materials

    from . import batch as bmod
    imgs = batch_specimens(a.count, l_max=a.max_side)
    k, e, m = two_phase_materials()
    bt = bmod.Batch(imgs, k, e, m, dt=0.01, damping=0.1, precision=a.precision)
    bt.set_schedule(a.tile_y, 0, 1)
    t0 = time.perf_counter()
    for i in range(1, a.increments + 1):
        bt.apply_strain(i * a.eps_inc)
        bt.step(a.steps)
    bt.synchronize()
    dt = time.perf_counter() - t0
    out = {"case": "batch", "specimens": len(imgs), "springs": int(sum(mm for _, mm in bt.sizes)),
           "seconds": dt, "last_sample_0": bt.samples(0)[-1], "kernel_launches": bt.counters()[1]}
    bt.close()
    return out


def _unet(a):
    import numpy as np
    import torch

    from . import nn
    net = nn.UNet(a.side, a.side, a.batch, seed=a.seed)
    rng = np.random.default_rng(a.seed)
    x = np.zeros((a.batch, a.side, a.side, 32), np.float32)
    x[..., :7] = rng.standard_normal((a.batch, a.side, a.side, 7))
    tx = torch.from_numpy(x).to(torch.bfloat16).cuda()
    tt = torch.from_numpy(rng.standard_normal((a.batch, a.side, a.side, 2)).astype(np.float32)).cuda()
    t0 = time.perf_counter()
    losses = [net.train_step(tx, tt, a.batch, 1e-3) for _ in range(a.iters)]
    torch.cuda.synchronize()
    out = {"case": "unet", "side": a.side, "batch": a.batch, "iters": a.iters, "seconds": time.perf_counter() - t0,
           "loss_first": losses[0], "loss_last": losses[-1]}
    net.close()
    return out


# (Cin, Cout, level) of the U-Net's 3x3 convolutions, level l at side / 2^l
_UNET_CONVS = [(32, 32, 0), (32, 32, 0), (32, 64, 1), (64, 64, 1), (64, 128, 2), (128, 128, 2), (128, 256, 3),
               (256, 256, 3), (384, 128, 2), (128, 128, 2), (192, 64, 1), (64, 64, 1), (96, 32, 0), (32, 32, 0)]


def _conv(a):
    import torch

    from . import nn
    L = nn.lib()
    st = torch.cuda.current_stream()
    sh = C.c_void_p(st.cuda_stream)
    gen = torch.Generator(device="cuda").manual_seed(a.seed)
    rows = []
    tot = {"flop": 0.0}
    for q, (cin, cout, lev) in enumerate(_UNET_CONVS):
        if a.layer >= 0 and q != a.layer:
            continue
        H = W = a.side >> lev
        B = a.batch
        x = torch.randn((B, H, W, cin), device="cuda", generator=gen).to(torch.bfloat16)
        w = (torch.randn((cout, 9, cin), device="cuda", generator=gen) * 0.05).to(torch.bfloat16)
        g = torch.randn((B, H, W, cout), device="cuda", generator=gen).to(torch.bfloat16)
        bias = torch.zeros(cout, device="cuda")
        out = torch.empty((B, H, W, cout), device="cuda", dtype=torch.bfloat16)
        dW = torch.empty(cout * 9 * cin, device="cuda")
        db = torch.empty(cout, device="cuda")
        ws = torch.empty(max(1 << 22, 16 * cout * 9 * cin), device="cuda")

        def fwd():
            nn.check(L.lsm_nn_conv_forward(nn.ptr(x), cin, 0, cin, nn.ptr(w), nn.ptr(bias), nn.ptr(out), cout, 0,
                                           cout, B, H, W, 9, 1, sh))

        def wgrad():
            nn.check(L.lsm_nn_conv_wgrad(nn.ptr(g), cout, nn.ptr(x), cin, 0, cin, B, H, W, 9, nn.ptr(dW),
                                         nn.ptr(db), nn.ptr(ws), ws.numel(), sh))

        flop = 2.0 * B * H * W * cout * cin * 9
        row = {"conv": q, "cin": cin, "cout": cout, "side": H}
        for name, fn in (("fwd", fwd), ("wgrad", wgrad)):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(a.iters):
                fn()
            e1.record(st)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / a.iters
            row[name + "_ms"] = ms
            row[name + "_tflops"] = flop / ms * 1e-9
        tot["flop"] += flop
        rows.append(row)
    if not rows:
        raise SystemExit("--layer must be in 0..13")
    out = {"case": "conv", "side": a.side, "batch": a.batch, "iters": a.iters, "layers": rows,
           "note": "fwd_ms: one lsm_nn_conv_forward call, which synchronises to report a timed-out wait; "
                   "wgrad_ms: asynchronous calls back to back"}
    if a.layer < 0:
        # the whole network, asynchronous: forward, and a training step
        # (forward, data and weight gradients of every convolution, Adam)
        net = nn.UNet(a.side, a.side, a.batch, seed=a.seed)
        x = torch.zeros((a.batch, a.side, a.side, 32), device="cuda").to(torch.bfloat16)
        x[..., :7] = torch.randn((a.batch, a.side, a.side, 7), device="cuda", generator=gen).to(torch.bfloat16)
        tt = torch.randn((a.batch, a.side, a.side, 2), device="cuda", generator=gen)
        pred = torch.empty((a.batch, a.side, a.side, 2), device="cuda")
        # training: forward, weight gradient and data gradient of every
        # convolution but the first (the input needs no gradient)
        f0 = 2.0 * a.batch * a.side * a.side * 32 * 32 * 9
        for name, fn, flop in (("forward", lambda: net.forward(x, pred, a.batch), tot["flop"]),
                               ("train_step", lambda: net.train_step(x, tt, a.batch, 1e-4, want_loss=False),
                                3.0 * tot["flop"] - f0)):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(a.iters):
                fn()
            e1.record(st)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / a.iters
            out["net_" + name + "_ms"] = ms
            out["net_" + name + "_conv_tflops"] = flop / ms * 1e-9
        net.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("case", choices=["single", "foam", "batch", "unet", "conv"])
    ap.add_argument("--side", type=int, default=256)
    ap.add_argument("--precision", default="df64", choices=["exact64", "fast64", "f32", "df64"])
    ap.add_argument("--path", type=int, default=0, choices=[0, 1, 2, 3],
                    help="single, foam: 0 automatic (tile and strip kernels), 1 spring-list kernels, "
                         "2 (single) tile kernel for every step, 3 (single) strip kernel for every step")
    ap.add_argument("--lattice", type=int, default=0, choices=[0, 1],
                    help="single: 0 square lattice, 1 the paper's triangular packing")
    ap.add_argument("--increments", type=int, default=3)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--eps-inc", type=float, default=1e-3)
    ap.add_argument("--rate", action="store_true",
                    help="single: after the first increment, grips at a constant strain rate instead of increments")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--count", type=int, default=64, help="batch: number of specimens")
    ap.add_argument("--max-side", type=int, default=512, help="batch: largest specimen side")
    ap.add_argument("--tile-y", type=int, default=16, help="batch: tile height (8, 16 or 32), or -8, -16, -32 for strips")
    ap.add_argument("--batch", type=int, default=8, help="unet: batch size")
    ap.add_argument("--iters", type=int, default=3, help="unet: training iterations; conv: timed calls per layer")
    ap.add_argument("--layer", type=int, default=-1, help="conv: only this convolution (0..13)")
    a = ap.parse_args(argv)
    out = {"single": _single, "foam": _foam, "batch": _batch, "unet": _unet, "conv": _conv}[a.case](a)
    print(json.dumps(out, default=float))
    return 0


if __name__ == "__main__":
    sys.exit(main())
