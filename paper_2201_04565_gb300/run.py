"""Command-line runs of the lattice-spring path on seeded synthetic specimens.

  python -m paper_2201_04565_gb300.run single --side 2048 --precision df64 --increments 3
  python -m paper_2201_04565_gb300.run foam --side 96 --precision df64 --increments 3
  python -m paper_2201_04565_gb300.run batch --count 64 --precision df64 --increments 3
  python -m paper_2201_04565_gb300.run unet --side 256 --batch 8 --iters 3

single: a 2D two-phase inclusion composite (fused tile kernel, or the
spring-list kernels with --path 1); foam: a 3D one-phase foam under
compression (voxel tile kernel in df64 / f32, spring-list kernels in the FP64
modes or with --path 1); batch: uneven 2D specimens (sides 32 to
--max-side) in one batched context; unet: training iterations of the
warm-start network on random inputs. Each case runs a displacement-controlled
tension (or compression) test of --increments load increments of --steps time
steps and prints a one-line JSON summary (last stress sample, broken springs,
kernel launches).
"""
from __future__ import annotations

import argparse
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
    for i in range(1, a.increments + 1):
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


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("case", choices=["single", "foam", "batch", "unet"])
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
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--count", type=int, default=64, help="batch: number of specimens")
    ap.add_argument("--max-side", type=int, default=512, help="batch: largest specimen side")
    ap.add_argument("--tile-y", type=int, default=16, help="batch: tile height (8, 16 or 32)")
    ap.add_argument("--batch", type=int, default=8, help="unet: batch size")
    ap.add_argument("--iters", type=int, default=3, help="unet: training iterations")
    a = ap.parse_args(argv)
    out = {"single": _single, "foam": _foam, "batch": _batch, "unet": _unet}[a.case](a)
    print(json.dumps(out, default=float))
    return 0


if __name__ == "__main__":
    sys.exit(main())
