"""Learned warm start: data generation, training and the curves/s comparison.

Every step of the method and of the network runs in liblsm's kernels; this
module only sequences the calls and holds device buffers (torch tensors are
used as plain storage and for device-to-device copies of whole samples).

One training sample is one strain increment of one specimen:
  input   phase map, displacement before the increment, strain before it,
          and the increment (lsm_unet_prepare_input);
  target  what the damped relaxation adds after the affine load step,
          u_relaxed - u_loaded (lsm_unet_prepare_target).
At use, the prediction is added to the loaded state before the relaxation
(lsm_batch_add_displacements); the relaxation then runs to the usual
force-residual tolerance, so the result of an increment without breaks does
not depend on the network (to that tolerance). Breaks are tested at every
step of the relaxation, so where springs break the changed transient can
change which of them break; the comparison records each arm's outcome
(stresses, broken springs, first breaks) beside its cost.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np

from . import batch as bmod
from . import lsm
from . import nn as nnmod

RELAX = dict(dt=0.5, damping=0.03)  # damped-dynamics relaxation settings (see the design notes)


def _torch():
    import torch
    return torch


def _stream():
    """The caller's current torch stream: every library object and call in this
    module is ordered on it, so torch's copies into and out of the shared
    buffers are ordered with the library's kernels."""
    return lsm.torch_stream_handle()


def _sp():
    import ctypes
    return ctypes.c_void_p(_stream())


_WORK = None


def _on_work_stream(fn):
    """Run fn with a dedicated torch stream as the current stream (the step
    loops are CUDA graphs, which cannot be captured on the legacy default
    stream), then wait for it."""
    import functools

    @functools.wraps(fn)
    def wrapped(*args, **kw):
        global _WORK
        torch = _torch()
        if _WORK is None:
            _WORK = torch.cuda.Stream()
        _WORK.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(_WORK):
            out = fn(*args, **kw)
        torch.cuda.current_stream().wait_stream(_WORK)
        _WORK.synchronize()
        return out
    return wrapped


class Fields:
    """Device buffers for S equal-size specimens."""

    def __init__(self, S, H, W):
        torch = _torch()
        self.S, self.H, self.W = S, H, W
        self.u = torch.empty((S, 2, H, W), dtype=torch.float32, device="cuda")
        self.phase = torch.empty((S, H, W), dtype=torch.uint8, device="cuda")

    def read(self, bt, with_phase=False):
        nnmod.check(nnmod.lib().lsm_batch_fields(bt.h, nnmod.ptr(self.u), nnmod.ptr(self.phase) if with_phase else None,
                                                 self.H, self.W), bt.h, batch=True)


def save_params(net, path):
    """Network parameters (FP32 master copy, .npy): the convolutions use
    their BF16 rounding, the biases and the head use them as they are."""
    np.save(path, net.get_params().astype(np.float32))


def load_params(net, path):
    """Parameters from save_params; a uint16 file holds BF16 bit patterns
    (an earlier format, which rounds the biases and the head too)."""
    p = np.load(path)
    if p.dtype == np.uint16:
        p = (p.astype(np.uint32) << 16).view(np.float32)
    net.set_params(p.astype(np.float32))


@_on_work_stream
def generate(images, k, e, m, increments, deps=1e-3, tol=1e-6, max_steps=200000, check_every=50,
             precision="f32", log=None, pre_fracture=False):
    """Run every specimen through `increments` load increments with the batched
    relaxation and return the samples on the device:
    U [N][2][H][W] (displacement before), phase [S][H][W], spec [N] (specimen
    index of each sample), eps [N] (strain before), T [N][H][W][2] (target).
    pre_fracture: keep only the increments that end with no broken spring in
    their specimen (the model the gated warm start uses)."""
    torch = _torch()
    S = len(images)
    H, W = images[0].shape
    bt = bmod.Batch(images, k, e, m, precision=precision, stream=_stream(), **RELAX)
    f = Fields(S, H, W)
    f.read(bt, with_phase=True)
    phase = f.phase.clone()
    N = S * increments
    U = torch.empty((N, 2, H, W), dtype=torch.float32, device="cuda")
    T = torch.empty((N, H, W, 2), dtype=torch.float32, device="cuda")
    spec = torch.arange(N, device="cuda", dtype=torch.int64) % S
    eps_b = torch.empty(N, dtype=torch.float32, device="cuda")
    loaded = torch.empty_like(f.u)
    intact = torch.ones(N, dtype=torch.bool, device="cuda")
    steps = []
    t0 = time.perf_counter()
    for i in range(increments):
        eps0 = i * deps
        f.read(bt)
        U[i * S:(i + 1) * S].copy_(f.u)
        eps_b[i * S:(i + 1) * S] = eps0
        bt.apply_strain((i + 1) * deps)
        f.read(bt)
        loaded.copy_(f.u)
        st, taken, conv = bt.relax(tol, max_steps, check_every)
        steps.append(int(np.mean(taken)))
        f.read(bt)
        nnmod.check(nnmod.lib().lsm_unet_prepare_target(nnmod.ptr(loaded), nnmod.ptr(f.u), deps, S, H, W, 1.0,
                                                        nnmod.ptr(T[i * S:(i + 1) * S]), _sp()))
        if log:
            log("increment %d: mean steps %d, converged %d/%d, %.1fs" % (i + 1, steps[-1], conv.sum(), S,
                                                                         time.perf_counter() - t0))
        if pre_fracture:
            intact[i * S:(i + 1) * S] = torch.tensor([bt.broken(q)[1] < 0 for q in range(S)], device="cuda")
    torch.cuda.synchronize()
    bt.close()
    if pre_fracture:
        keep = torch.nonzero(intact).flatten()
        U, T, spec, eps_b = U[keep].contiguous(), T[keep].contiguous(), spec[keep].contiguous(), eps_b[keep].contiguous()
    return dict(U=U, T=T, phase=phase, spec=spec, eps=eps_b, deps=deps, H=H, W=W, steps=steps,
                seconds=time.perf_counter() - t0)


@_on_work_stream
def train(data, steps=2000, batch=16, lr=1e-3, seed=0, log=None, val=None):
    """Adam on the mean squared error over random minibatches of samples."""
    torch = _torch()
    H, W = data["H"], data["W"]
    net = nnmod.UNet(H, W, batch, seed=seed, stream=_stream())
    N = data["U"].shape[0]
    rng = np.random.default_rng(seed)
    xb = torch.empty((batch, H, W, 32), dtype=torch.bfloat16, device="cuda")
    ub = torch.empty((batch, 2, H, W), dtype=torch.float32, device="cuda")
    pb = torch.empty((batch, H, W), dtype=torch.uint8, device="cuda")
    eb = torch.empty(batch, dtype=torch.float32, device="cuda")
    tb = torch.empty((batch, H, W, 2), dtype=torch.float32, device="cuda")
    hist = []
    t0 = time.perf_counter()
    for it in range(steps):
        idx = torch.from_numpy(rng.integers(0, N, size=batch)).cuda()
        torch.index_select(data["U"], 0, idx, out=ub)
        torch.index_select(data["phase"], 0, data["spec"][idx], out=pb)
        torch.index_select(data["eps"], 0, idx, out=eb)
        torch.index_select(data["T"], 0, idx, out=tb)
        nnmod.check(nnmod.lib().lsm_unet_prepare_input(nnmod.ptr(pb), nnmod.ptr(ub), nnmod.ptr(eb), data["deps"],
                                                       batch, H, W, 1.0, nnmod.ptr(xb), _sp()))
        cur = lr * 0.5 * (1.0 + math.cos(math.pi * it / steps))  # cosine decay
        want = it % 100 == 0 or it == steps - 1
        loss = net.train_step(xb, tb, batch, cur, want_loss=want)
        if want:
            hist.append((it, loss))
            if log:
                log("train step %d loss %.4e lr %.2e (%.1fs)" % (it, loss, cur, time.perf_counter() - t0))
    torch.cuda.synchronize()
    return net, dict(loss_history=hist, seconds=time.perf_counter() - t0, steps=steps, batch=batch)


@_on_work_stream
def relative_error(net, data, batch=16):
    """Normwise relative error of the prediction over a data set (target
    units): ||pred - target|| / ||target||."""
    torch = _torch()
    H, W = data["H"], data["W"]
    N = data["U"].shape[0]
    xb = torch.empty((batch, H, W, 32), dtype=torch.bfloat16, device="cuda")
    out = torch.empty((batch, H, W, 2), dtype=torch.float32, device="cuda")
    num = den = 0.0
    for s0 in range(0, N - batch + 1, batch):
        sl = slice(s0, s0 + batch)
        ph = data["phase"][data["spec"][sl]].contiguous()
        nnmod.check(nnmod.lib().lsm_unet_prepare_input(nnmod.ptr(ph), nnmod.ptr(data["U"][sl].contiguous()),
                                                       nnmod.ptr(data["eps"][sl].contiguous()), data["deps"], batch,
                                                       H, W, 1.0, nnmod.ptr(xb), _sp()))
        net.forward(xb, out, batch)
        t = data["T"][sl]
        num += float(((out - t) ** 2).sum())
        den += float((t ** 2).sum())
    return math.sqrt(num / max(den, 1e-300))


def _predict_du(net, f, bt, eps_before, deps, xb, out, du, chunk):
    """Prediction of every specimen's relaxation displacement, in chunks of the
    network's batch size, written into du [S][2][H][W]."""
    torch = _torch()
    S, H, W = f.S, f.H, f.W
    eps_t = torch.full((S,), eps_before, dtype=torch.float32, device="cuda")
    for s0 in range(0, S, chunk):
        n = min(chunk, S - s0)
        nnmod.check(nnmod.lib().lsm_unet_prepare_input(nnmod.ptr(f.phase[s0:s0 + n]), nnmod.ptr(f.u[s0:s0 + n]),
                                                       nnmod.ptr(eps_t[s0:s0 + n]), deps, n, H, W, 1.0,
                                                       nnmod.ptr(xb), _sp()))
        net.forward(xb, out, n)
        nnmod.check(nnmod.lib().lsm_unet_prediction_to_displacement(nnmod.ptr(out), deps, n, H, W, 1.0,
                                                                    nnmod.ptr(du[s0:s0 + n]), _sp()))


@_on_work_stream
def compare(images, k, e, m, net, first_inc, increments, deps=1e-3, tol=1e-8, max_steps=400000, check_every=50,
            precision="df64", plain_every=1, log=None, gate=True):
    """Wall time per increment of three arms on the same specimens, each run
    from the unloaded state through first_inc - 1 unmeasured increments, then
    `increments` measured ones, all relaxed to the same tolerance:
      plain    one single-specimen context per specimen, one after another;
      batched  all specimens in one lsm_batch;
      warm     batched, with the network's prediction added before relaxing
               (gate: only for specimens with no broken spring yet; after the
               first break the prediction slowed the relaxation down, see the
               design notes).
    Returns per-arm seconds and steps."""
    torch = _torch()
    S = len(images)
    H, W = images[0].shape
    res = {}

    # batched and warm-started arms
    for arm in ("batched", "warm"):
        bt = bmod.Batch(images, k, e, m, precision=precision, stream=_stream(), **RELAX)
        f = Fields(S, H, W)
        f.read(bt, with_phase=True)
        chunk = net.max_batch if net is not None else 1
        xb = torch.empty((chunk, H, W, 32), dtype=torch.bfloat16, device="cuda")
        out = torch.empty((chunk, H, W, 2), dtype=torch.float32, device="cuda")
        du = torch.empty((S, 2, H, W), dtype=torch.float32, device="cuda")
        times, steps, nconv, sig = [], [], 0, []
        for i in range(1, first_inc + increments):
            measured = i >= first_inc
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if arm == "warm":
                f.read(bt)  # state before the increment
                _predict_du(net, f, bt, (i - 1) * deps, deps, xb, out, du, chunk)
            bt.apply_strain(i * deps)
            if arm == "warm":
                if gate:  # no prediction for specimens that have started to fracture
                    for q in range(S):
                        if bt.broken(q)[1] >= 0:
                            du[q].zero_()
                nnmod.check(nnmod.lib().lsm_batch_add_displacements(bt.h, nnmod.ptr(du), H, W), bt.h, batch=True)
            st, taken, conv = bt.relax(tol, max_steps, check_every)
            torch.cuda.synchronize()
            if measured:
                times.append(time.perf_counter() - t0)
                steps.append(taken.tolist())
                nconv += int(conv.sum())
                # outcome, outside the timed region: each specimen's stress
                sig.append([bt.samples(q)[-1]["sigma_vir"] for q in range(S)])
                if log:
                    log("%s increment %d: %.2fs, mean steps %d" % (arm, i, times[-1], int(np.mean(taken))))
        brk = [bt.broken(q) for q in range(S)]
        res[arm] = dict(seconds=times, steps_mean=[float(np.mean(s)) for s in steps],
                        steps_max=[int(np.max(s)) for s in steps], converged=nconv, of=S * increments,
                        sigma=sig, n_broken=[int(b[0].sum()) for b in brk], first_break=[int(b[1]) for b in brk])
        bt.close()
    # plain arm: one context per specimen (every plain_every-th specimen, scaled)
    sub = list(range(0, S, plain_every))
    tot = [0.0] * increments
    st_inc = [[] for _ in range(increments)]
    p_sig, p_brk, p_fb, p_conv = [[] for _ in range(increments)], [], [], 0
    for q in sub:
        sp = lsm.Specimen.from_image(images[q], k, e, m, precision=precision, stream=_stream(), **RELAX)
        for i in range(1, first_inc + increments):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sp.apply_strain(i * deps)
            stq, taken = sp.relax(tol, max_steps, check_every)
            torch.cuda.synchronize()
            if i >= first_inc:
                tot[i - first_inc] += time.perf_counter() - t0
                st_inc[i - first_inc].append(taken)
                p_conv += int(stq == lsm.LSM_OK)
                p_sig[i - first_inc].append(sp.last_sample()["sigma_vir"])
        b = sp.broken()
        p_brk.append(int(b[0].sum()))
        p_fb.append(int(b[1]))
        sp.close()
    scale = S / len(sub)
    res["plain"] = dict(seconds=[t * scale for t in tot], steps_mean=[float(np.mean(q)) for q in st_inc],
                        steps_max=[int(np.max(q)) for q in st_inc], converged=p_conv, of=len(sub) * increments,
                        sigma=p_sig, n_broken=p_brk, first_break=p_fb,
                        sample="%d of %d specimens run, time scaled by the specimen count" % (len(sub), S))
    # a curve = 100 increments (10% strain); with first_inc 1 and 100
    # measured increments every curve was run to its end (no extrapolation)
    res["full_curves"] = first_inc == 1 and increments >= 100
    for arm in ("plain", "batched", "warm"):
        per_inc = float(np.mean(res[arm]["seconds"]))
        res[arm]["seconds_per_increment"] = per_inc
        res[arm]["seconds_total"] = float(np.sum(res[arm]["seconds"]))
        res[arm]["curves_per_s"] = S / (per_inc * 100.0)
    res["speedup_warm_vs_plain"] = res["plain"]["seconds_per_increment"] / res["warm"]["seconds_per_increment"]
    res["speedup_batched_vs_plain"] = res["plain"]["seconds_per_increment"] / res["batched"]["seconds_per_increment"]
    res["speedup_warm_vs_batched"] = res["batched"]["seconds_per_increment"] / res["warm"]["seconds_per_increment"]
    return res


@_on_work_stream
def steps_to_tolerance(images, k, e, m, net, increments, deps=1e-3, tol=1e-8, max_steps=400000, check_every=50,
                       precision="df64", gate=True, log=None):
    """Steps the batched relaxation needs per increment, without the network
    (arm "batched") and with its prediction added after each load step (arm
    "warm"; gate: only for specimens with no broken spring yet), both to the
    same force-residual tolerance, from the unloaded state through
    `increments` increments. Returns per arm: steps [increment][specimen],
    converged flags, wall seconds per increment, the final positions of
    every specimen and its last sample."""
    torch = _torch()
    S = len(images)
    H, W = images[0].shape
    res = {}
    for arm in ("batched", "warm"):
        bt = bmod.Batch(images, k, e, m, precision=precision, stream=_stream(), **RELAX)
        f = Fields(S, H, W)
        f.read(bt, with_phase=True)
        chunk = net.max_batch
        xb = torch.empty((chunk, H, W, 32), dtype=torch.bfloat16, device="cuda")
        out = torch.empty((chunk, H, W, 2), dtype=torch.float32, device="cuda")
        du = torch.empty((S, 2, H, W), dtype=torch.float32, device="cuda")
        steps, conv_all, secs = [], [], []
        for i in range(1, increments + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if arm == "warm":
                f.read(bt)  # state before the increment
                _predict_du(net, f, bt, (i - 1) * deps, deps, xb, out, du, chunk)
            bt.apply_strain(i * deps)
            if arm == "warm":
                if gate:
                    for q in range(S):
                        if bt.broken(q)[1] >= 0:
                            du[q].zero_()
                nnmod.check(nnmod.lib().lsm_batch_add_displacements(bt.h, nnmod.ptr(du), H, W), bt.h, batch=True)
            st, taken, conv = bt.relax(tol, max_steps, check_every)
            torch.cuda.synchronize()
            secs.append(time.perf_counter() - t0)
            steps.append([int(t) for t in taken])
            conv_all.append([bool(c) for c in conv])
            if log:
                log("%s increment %d: %.2fs, steps %d (mean)" % (arm, i, secs[-1], int(np.mean(taken))))
        res[arm] = dict(steps=steps, converged=conv_all, seconds=secs,
                        x=[bt.state(q)[0] for q in range(S)], last=[bt.samples(q)[-1] for q in range(S)],
                        first_break=[bt.broken(q)[1] for q in range(S)])
        bt.close()
    return res


def main(argv=None):
    """End-to-end: generate, train, validate, compare; prints one JSON line."""
    import argparse
    import sys

    from gen.images import two_phase_materials, warmstart_specimens

    ap = argparse.ArgumentParser()
    ap.add_argument("--side", type=int, default=256)
    ap.add_argument("--train-specimens", type=int, default=200)
    ap.add_argument("--train-increments", type=int, default=100)
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--val-specimens", type=int, default=16)
    ap.add_argument("--val-increments", type=int, default=5)
    ap.add_argument("--eval-specimens", type=int, default=256)
    ap.add_argument("--eval-first", type=int, default=1)
    ap.add_argument("--eval-increments", type=int, default=2)
    ap.add_argument("--plain-every", type=int, default=8)
    ap.add_argument("--data-tol", type=float, default=1e-6)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--check-every", type=int, default=50, help="comparison: residual checked every n steps")
    ap.add_argument("--pre-fracture", action="store_true",
                    help="train on the increments that end before their specimen's first break")
    ap.add_argument("--data-precision", default="f32", choices=["f32", "df64"])
    ap.add_argument("--save", default=None)
    ap.add_argument("--load", default=None, help="skip training: BF16 weights from save_params")
    a = ap.parse_args(argv)

    def log(msg):
        sys.stderr.write(msg + "\n")
        sys.stderr.flush()

    k, e, m = two_phase_materials()
    train_imgs = [] if a.load else warmstart_specimens(range(a.train_specimens), side=a.side)
    val_imgs = warmstart_specimens(range(2000, 2000 + a.val_specimens), side=a.side)
    vdata = generate(val_imgs, k, e, m, a.val_increments, tol=a.data_tol, log=log, precision=a.data_precision,
                     pre_fracture=a.pre_fracture)
    if a.load:
        net = nnmod.UNet(a.side, a.side, 16, stream=_stream())
        load_params(net, a.load)
        data = dict(U=vdata["U"][:0], seconds=0.0, steps=[0])
        tinfo, terr = dict(loaded=a.load), float("nan")
    else:
        data = generate(train_imgs, k, e, m, a.train_increments, tol=a.data_tol, log=log,
                        precision=a.data_precision, pre_fracture=a.pre_fracture)
        net, tinfo = train(data, steps=a.train_steps, log=log)
        terr = relative_error(net, {**data, "U": data["U"][:512], "T": data["T"][:512],
                                    "spec": data["spec"][:512], "eps": data["eps"][:512]})
    verr = relative_error(net, vdata)
    log("relative prediction error: train %.3f, held-out %.3f" % (terr, verr))
    if a.save:
        save_params(net, a.save)
    eval_imgs = warmstart_specimens(range(1000, 1000 + a.eval_specimens), side=a.side)
    cmp = compare(eval_imgs, k, e, m, net, a.eval_first, a.eval_increments, tol=a.tol, plain_every=a.plain_every,
                  check_every=a.check_every, log=log)
    out = dict(workload="warmstart_%dx%d_x%d" % (a.side, a.side, a.eval_specimens),
               data=dict(samples=int(data["U"].shape[0]), specimens=a.train_specimens,
                         increments=a.train_increments, tol=a.data_tol, seconds=data["seconds"],
                         mean_steps_per_increment=float(np.mean(data["steps"]))),
               training=dict(tinfo, train_rel_error=terr, heldout_rel_error=verr),
               comparison=cmp)
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    import sys
    sys.exit(main())
