#!/usr/bin/env python3
"""Benchmark of the lattice-spring hot path on one GB300 (or N replicas).

One bench step = one displacement-controlled load increment of the 2D
2048 x 2048 two-phase composite (4,194,304 particles, 16,764,930 springs):
lsm_apply_strain, 20 damped velocity-Verlet time steps with the break test,
and the stress sample. The metric is spring-updates/s (springs x time steps
per second), whole job over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision MODE]
  python bench.py --impl reference ...   # the FP64 CPU oracle, timed on the host

Under torchrun every rank steps its own replica of the specimen (the
single-specimen path does not shard; replicas only), timing is max over
ranks after a barrier, and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from gen.images import inclusion_image, two_phase_materials  # noqa: E402

WORKLOAD = dict(name="2d_2048_two_phase", nx=2048, ny=2048, r=(10.0, 60.0), frac=0.30, seed=1,
                dt=0.01, damping=0.1, steps_per_increment=20, eps_inc=1e-3)
METRIC = "spring-updates/sec (% HBM roofline) at 1 GB300"
UNIT = "spring-updates/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)  # let the sampler start before the timed region
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [q.strip() for q in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[5 + q].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def algorithmic_bytes(n, m, dim):
    """Bytes a general spring-network step must move: positions and half-step
    velocities read and written in FP64 (32 d bytes per particle) plus one
    10-byte spring record per spring (2 x int32 endpoints, type, state)."""
    return n * 32 * dim + 10 * m


# DRAM traffic of one time-step launch of each mode's 2D kernel on the
# 2048 x 2048 workload, from ncu (dram__bytes_read.sum + dram__bytes_write.sum),
# keyed by precision mode, with the sha1 prefix of the kernel source it was
# taken on; once the kernel changes, traffic reports null until re-measured.
NCU_TRAFFIC = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum on three
    # time-step launches of each mode (the same 2048 x 2048 workload), mean
    "df64": (238.3e6, "5ebefc3dec19"),
    "f32": (240.1e6, "5ebefc3dec19"),
    "fast64": (236.2e6, "5ebefc3dec19"),
    "exact64": (236.9e6, "5ebefc3dec19"),
}

# Warp instructions executed by one time-step launch (ncu smsp__inst_executed.sum,
# same workload and kernel tag as NCU_TRAFFIC): with the issue peak of the
# part (152 SMs x 4 schedulers x 1 warp instruction per cycle at the SM clock)
# this gives the instruction-issue roofline, the one the fixed-point modes
# are bound by.
NCU_INSTRUCTIONS = {
    "df64": (108821973, "5ebefc3dec19"),
    "f32": (75982754, "5ebefc3dec19"),
    "fast64": (94464248, "5ebefc3dec19"),
    "exact64": (195572908, "5ebefc3dec19"),
}

# Binding unit of each mode's time-step kernel, from ncu on the same workload
# (see the profile summaries), for the roofline's "limiter" note.
LIMITER = {
    "df64": "instruction issue (ncu: 74% of issue slots busy, FP64 pipe 48%, DRAM 24% of peak)",
    "f32": "instruction issue (ncu: 72% of issue slots busy, FP64 pipe 52%, DRAM 33% of peak)",
    "fast64": "FP64 pipe (ncu: 86% busy)",
    "exact64": "FP64 pipe (ncu: 88% busy; correctly rounded sqrt and divide)",
}

# Time-step kernel of each mode on the 2D image lattice.
KERNEL = {
    "df64": "k_strip2d (register-resident strip kernel, one launch per time step)",
    "f32": "k_strip2d (register-resident strip kernel, one launch per time step)",
    "fast64": "k_tile2d (tile kernel, one launch per time step)",
    "exact64": "k_tile2d (tile kernel, one launch per time step)",
}


def _kernel_tag():
    """sha1 prefix of the 2D time-step kernels' sources (the strip kernel of
    the fixed-point modes and its sweep, the tile kernel of the FP64 modes,
    and the arithmetic they share)."""
    import hashlib
    h = hashlib.sha1()
    for name in ("strip2d.cu", "strip_body.cuh", "tile2d.cu", "tile_body.cuh", "dfloat.cuh"):
        with open(os.path.join(ROOT, "paper_2201_04565_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def _issue_roofline(precision, launch_ms, clk):
    """Issue rate of the time-step kernel against the part's issue peak
    (152 SMs x 4 warp schedulers x one warp instruction per cycle at the SM
    clock seen during the run), from the ncu instruction count of the same
    kernel source; None when no count matches the current source."""
    if precision not in NCU_INSTRUCTIONS or NCU_INSTRUCTIONS[precision][1] != _kernel_tag():
        return None
    inst = NCU_INSTRUCTIONS[precision][0]
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    peak = 152 * 4 * mhz * 1e6
    achieved = inst / (launch_ms * 1e-3)
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "warp instructions/s",
            "frac": achieved / peak, "instructions_per_launch": inst,
            "peak_source": "152 SMs x 4 schedulers x 1 warp instruction/cycle x %.0f MHz (sampled)" % mhz}


def _build_specimen(lsm, precision, stream):
    img = inclusion_image(WORKLOAD["nx"], WORKLOAD["ny"], *WORKLOAD["r"], WORKLOAD["frac"], WORKLOAD["seed"])
    k, e, m = two_phase_materials()
    return lsm.Specimen.from_image(img, k, e, m, dt=WORKLOAD["dt"], damping=WORKLOAD["damping"],
                                   precision=precision, stream=stream.cuda_stream)


def _time_increments(spec, stream, first_inc, count):
    """Events around every lsm_step (one increment = nst time steps) on the
    library's stream; returns (total ms, per-increment ms list)."""
    import torch
    nst = WORKLOAD["steps_per_increment"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(count)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for q in range(count):
        spec.apply_strain((first_inc + q) * WORKLOAD["eps_inc"])
        ev[q][0].record(stream)
        spec.step(nst)
        ev[q][1].record(stream)
    t1.record(stream)
    stream.synchronize()
    return t0.elapsed_time(t1), [a.elapsed_time(b) for a, b in ev]


def run_gpu(args, rank, world):
    import torch
    from paper_2201_04565_gb300 import lsm

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    spec = _build_specimen(lsm, args.precision, stream)
    nst = WORKLOAD["steps_per_increment"]
    inc = 0
    for _ in range(args.warmup):
        inc += 1
        spec.apply_strain(inc * WORKLOAD["eps_inc"])
        spec.step(nst)
    spec.synchronize()
    dist = world > 1
    if dist:
        import torch.distributed as td
        td.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    launches0 = spec.counters()[2]
    ms, inc_ms = _time_increments(spec, stream, inc + 1, args.steps)
    inc += args.steps
    torch.cuda.synchronize()
    launches = spec.counters()[2] - launches0
    clk = clocks.stop()
    if dist:
        import torch.distributed as td
        t = torch.tensor([ms], device="cuda")
        td.all_reduce(t, op=td.ReduceOp.MAX)
        ms = float(t.item())
        td.barrier()

    # end to end through the public API with host buffers: the strain goes in
    # from the host, every increment's stress sample and broken-spring mask
    # come back into page-locked host memory (two sets, alternating) through
    # the pipelined readback, whose copies overlap the next increment's steps;
    # the timed region ends when the last copy has landed
    e2e_steps = max(3, min(args.steps, 10))
    mask_host = [torch.empty(max(spec.m, 1), dtype=torch.uint8, pin_memory=True).numpy() for _ in range(2)]
    sample_host = [torch.empty(64, dtype=torch.uint8, pin_memory=True).numpy() for _ in range(2)]
    spec.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        inc += 1
        spec.apply_strain(inc * WORKLOAD["eps_inc"])
        spec.step(nst)
        spec.readback_async(mask_host[k % 2], sample_host[k % 2])
    spec.readback_wait()
    t1 = time.perf_counter()
    last = (e2e_steps - 1) % 2
    assert lsm.sample_from_buffer(sample_host[last])["step"] == inc * nst
    assert np.array_equal(mask_host[last][:spec.m], spec.broken()[0])
    e2e_value = spec.m * nst * e2e_steps * world / (t1 - t0)
    d2h = spec.m + 64  # broken mask + the increment's sample (one 64-byte record)

    hbm, peak_src = _peaks()
    units = spec.m * nst * args.steps * world
    value = units / (ms * 1e-3)
    # one time step = one launch of the fused tile kernel; the increment's
    # events also cover the sample reduction (one tiny kernel), so this
    # slightly overstates the kernel's duration
    per_step_ms = statistics.mean(inc_ms) / nst
    algb = algorithmic_bytes(spec.n, spec.m, spec.dim)
    achieved = algb / (per_step_ms * 1e-3) / 1e9
    traffic = None
    if args.precision in NCU_TRAFFIC and NCU_TRAFFIC[args.precision][1] == _kernel_tag():
        traffic = NCU_TRAFFIC[args.precision][0]
    dtype = {"exact64": "f64", "fast64": "f64", "f32": "f32 force / f64 state",
             "df64": "f32x2 (double-float) force / f64 state"}[args.precision]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic (seeded two-phase inclusion image; the paper's specimen files are not used)",
        "config": _config_2d(spec.n, spec.m, spec.dim, args.precision, world),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "kernel": KERNEL.get(args.precision),
                     "algorithmic_bytes_per_launch": algb, "launch_ms": per_step_ms,
                     "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)",
                     "limiter": LIMITER.get(args.precision)},
        "issue_roofline": _issue_roofline(args.precision, per_step_ms, clk),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8, "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    spec.close()

    if not args.no_variants and world == 1:
        variants = {}
        for mode in ("exact64", "fast64", "f32", "df64"):
            if mode == args.precision:
                variants[mode] = {"value": value, "time_step_ms": per_step_ms, "clocks": clk}
                continue
            sp = _build_specimen(lsm, mode, stream)
            for q in range(1, 4):
                sp.apply_strain(q * WORKLOAD["eps_inc"])
                sp.step(nst)
            sp.synchronize()
            vclk = ClockSampler(dev)
            vclk.start()
            vm, vinc = _time_increments(sp, stream, 4, 10)
            variants[mode] = {"value": sp.m * nst * 10 / (vm * 1e-3), "time_step_ms": statistics.mean(vinc) / nst,
                              "increments_timed": 10, "clocks": vclk.stop()}
            sp.close()
        out["variants"] = variants
    return out


def run_curves_subset(args, stride=4, incs=80, nst=20):
    """Converged stress-strain curves per second on a fixed subset of the
    512-specimen batch (every stride-th specimen of the seeded set: sides
    32..512 px, 10-50% inclusions), tension to 8% strain in 80 increments of
    20 time steps. Batched arm: one lsm_batch for the whole subset (one
    tile-kernel launch per time step for all specimens, graph-captured,
    autotuned schedule). Plain arm: one single-specimen context per
    specimen, run one after another. Both arms are timed through the API on
    the host clock, per-increment host work included, build and autotuning
    excluded; every specimen of the subset runs in both arms (nothing is
    extrapolated)."""
    import torch
    from gen.images import batch_specimens
    from paper_2201_04565_gb300 import batch as bmod
    from paper_2201_04565_gb300 import lsm
    prec = args.precision
    imgs = batch_specimens(512)[::stride]
    k, e, m = two_phase_materials()
    stream = torch.cuda.Stream()
    bt = bmod.Batch(imgs, k, e, m, dt=0.01, damping=0.1, precision=prec, stream=stream.cuda_stream)
    msum = sum(mm for _, mm in bt.sizes)
    t0 = time.perf_counter()
    tune = bt.autotune(10)
    t_tune = time.perf_counter() - t0
    bt.synchronize()
    t0 = time.perf_counter()
    for i in range(1, incs + 1):
        bt.apply_strain(i * 1e-3)
        bt.step(nst)
    bt.synchronize()
    t_batch = time.perf_counter() - t0
    bt.close()
    t_plain = 0.0
    for im in imgs:
        sp = lsm.Specimen.from_image(im, k, e, m, dt=0.01, damping=0.1, precision=prec,
                                     stream=stream.cuda_stream)
        sp.synchronize()
        t0 = time.perf_counter()
        for i in range(1, incs + 1):
            sp.apply_strain(i * 1e-3)
            sp.step(nst)
        sp.synchronize()
        t_plain += time.perf_counter() - t0
        sp.close()
    return {"metric": "converged stress-strain curves/s, batched vs plain per-specimen contexts",
            "workload": "batch512_two_phase subset: every %dth specimen (%d of 512), tension to %g%% strain"
                        % (stride, len(imgs), incs * 0.1),
            "specimens": len(imgs), "springs_total": msum, "increments": incs, "time_steps_per_increment": nst,
            "precision": prec,
            "batched": {"curves_per_s": len(imgs) / t_batch, "seconds": t_batch,
                        "spring_updates_per_s": msum * incs * nst / t_batch,
                        "schedule": tune, "autotune_seconds": t_tune},
            "plain": {"curves_per_s": len(imgs) / t_plain, "seconds": t_plain,
                      "spring_updates_per_s": msum * incs * nst / t_plain},
            "speedup": t_plain / t_batch,
            "warm_start": "not in this line: the learned warm start needs a network trained on "
                          "method-generated data (minutes of GPU time); measured separately"}


def run_batch512(args, rank=0, world=1, plain_every=8):
    """Uneven batch of 512 two-phase specimens (sides 32..512 px), tension to
    8% in 80 increments of 20 steps. Batched arm: every specimen in one
    lsm_batch (one tile-kernel launch per time step, graph-captured, autotuned
    schedule). Plain arm: one single-specimen context per specimen, run one
    after another through the same library (every plain_every-th specimen is
    run, and its time is scaled by the spring count of the whole batch).
    Build time is excluded from both arms; per-increment host work is
    included. Returns curves/s for both.

    Under torchrun the specimens are sharded across ranks (longest first to
    the lightest rank, by pixel count; no collective on the data path), each
    rank steps its share in its own batch, and the time is the maximum over
    ranks; the plain arm then runs on rank 0's share only."""
    import torch
    from gen.images import batch_specimens
    from paper_2201_04565_gb300 import batch as bmod
    from paper_2201_04565_gb300 import lsm
    from paper_2201_04565_gb300 import shard

    prec = args.precision
    imgs_all = batch_specimens(512)
    share = shard.my_share([im.size for im in imgs_all], rank, world)
    imgs = [imgs_all[q] for q in share]
    k, e, m = two_phase_materials()
    incs, nst = 80, 20
    stream = torch.cuda.Stream()
    bt = bmod.Batch(imgs, k, e, m, dt=0.01, damping=0.1, precision=prec, stream=stream.cuda_stream)
    msum = sum(mm for _, mm in bt.sizes)
    tune = bt.autotune(10)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as td
        td.barrier()
    t0 = time.perf_counter()
    for i in range(1, incs + 1):
        bt.apply_strain(i * 1e-3)
        bt.step(nst)
    bt.synchronize()
    t_batch = shard.max_over_ranks(time.perf_counter() - t0)
    launches = bt.counters()[1]
    bt.close()
    sub = list(range(0, len(imgs), plain_every))
    m_sub = 0
    t_plain = 0.0
    for q in sub:
        sp = lsm.Specimen.from_image(imgs[q], k, e, m, dt=0.01, damping=0.1, precision=prec,
                                     stream=stream.cuda_stream)
        m_sub += sp.m
        sp.synchronize()
        t0 = time.perf_counter()
        for i in range(1, incs + 1):
            sp.apply_strain(i * 1e-3)
            sp.step(nst)
        sp.synchronize()
        t_plain += time.perf_counter() - t0
        sp.close()
    t_plain_all = t_plain * msum / m_sub * world  # rank 0's share, scaled to the whole batch on one GPU
    return {"workload": "batch512_two_phase", "specimens": len(imgs_all), "n_gpus": world,
            "scaling": "strong" if world > 1 else "weak", "springs_total_rank0": msum,
            "increments": incs, "time_steps_per_increment": nst, "precision": prec,
            "batched": {"curves_per_s": len(imgs_all) / t_batch, "seconds": t_batch,
                        "spring_updates_per_s_rank0": msum * incs * nst / t_batch, "schedule_rank0": tune,
                        "kernel_launches_rank0": launches},
            "plain": {"curves_per_s": len(imgs_all) / t_plain_all, "seconds_extrapolated": t_plain_all,
                      "sample": "%d of rank 0's %d specimens run, time scaled by spring count%s"
                                % (len(sub), len(imgs), " and by the rank count" if world > 1 else "")},
            "speedup": t_plain_all / t_batch}


def run_foam256(args):
    """The 3D configuration: a 256^3 Gaussian-smoothed foam (35% solid, one
    phase, k = 1, critical strain 0.04), clamped grips, compression in 1e-3
    increments of 20 time steps. Same timing as the 2D workload (CUDA events
    on the library's stream around each lsm_step, after the warm-up
    increments); df64 and f32 run the voxel tile kernel, the FP64 modes the
    spring-list kernels."""
    import torch
    from gen.images import foam_volume, one_phase_materials
    from paper_2201_04565_gb300 import lsm
    stream = torch.cuda.Stream()
    img = foam_volume(256, 4.0, 0.35, seed=2)
    k, e, m = one_phase_materials(1.0, 0.04)
    sp = lsm.Specimen.from_image(img, k, e, m, dt=0.01, damping=0.1, precision=args.precision, grip_mode=1,
                                 stream=stream.cuda_stream)
    nst, inc = 20, 0
    for _ in range(args.warmup):
        inc += 1
        sp.apply_strain(-inc * 1e-3)
        sp.step(nst)
    sp.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    launches0 = sp.counters()[2]
    t0.record(stream)
    for _ in range(args.steps):
        inc += 1
        sp.apply_strain(-inc * 1e-3)
        sp.step(nst)
    t1.record(stream)
    stream.synchronize()
    ms = t0.elapsed_time(t1)
    hbm, peak_src = _peaks()
    algb = algorithmic_bytes(sp.n, sp.m, 3)
    per_step_ms = ms / (args.steps * nst)
    out = {"metric": METRIC, "value": sp.m * nst * args.steps / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic (seeded foam volume)",
           "config": {"workload": "3d_256_foam", "volume": "256^3", "particles": sp.n, "springs": sp.m,
                      "time_steps_per_bench_step": nst, "precision": args.precision,
                      "kernel": "k_tile3d" if args.precision in ("df64", "f32") else "k_springs + k_gather"},
           "roofline": {"bound": "hbm", "achieved": algb / (per_step_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": algb / (per_step_ms * 1e-3) / 1e9 / hbm, "traffic": None,
                        "algorithmic_bytes_per_launch": algb, "launch_ms": per_step_ms,
                        "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)"},
           "gpu_launches": int(sp.counters()[2] - launches0)}
    sp.close()
    return out


def run_next_rows(args):
    """The next rows of the scope on the 2048 x 2048 composite, one line
    each: the paper's triangular packing (lattice 1, spring-list kernels in
    the fixed-point modes: strip kernel on the packing's site grid), constant strain-rate loading of the grips (the
    tile kernel's rate instance; rate * dt * 20 = 1e-3 per 20 steps, as the
    increments of the main line), and the per-particle stress and strain
    fields (lsm_fields, particles per second). Same timing rules: warm-up
    first, CUDA events on the library's stream, inputs larger than L2."""
    import torch
    from paper_2201_04565_gb300 import lsm
    stream = torch.cuda.Stream()
    img = inclusion_image(WORKLOAD["nx"], WORKLOAD["ny"], *WORKLOAD["r"], WORKLOAD["frac"], WORKLOAD["seed"])
    k, e, m = two_phase_materials()
    nst = WORKLOAD["steps_per_increment"]
    hbm, peak_src = _peaks()
    out = {}

    def timed(spec, per_inc):
        for q in range(args.warmup):
            per_inc(q + 1)
        spec.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for q in range(args.steps):
            per_inc(args.warmup + q + 1)
        b.record(stream)
        stream.synchronize()
        return a.elapsed_time(b)

    def line(spec, ms, label, kernel):
        per_step = ms / (args.steps * nst)
        algb = algorithmic_bytes(spec.n, spec.m, 2)
        return {"value": spec.m * nst * args.steps / (ms * 1e-3), "unit": UNIT, "particles": spec.n,
                "springs": spec.m, "time_step_ms": per_step, "kernel": kernel,
                "roofline": {"bound": "hbm", "achieved": algb / (per_step * 1e-3) / 1e9, "peak": hbm,
                             "unit": "GB/s", "frac": algb / (per_step * 1e-3) / 1e9 / hbm,
                             "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)"},
                "workload": label}

    tri = lsm.Specimen.from_image(img, k, e, m, dt=WORKLOAD["dt"], damping=WORKLOAD["damping"],
                                  precision=args.precision, lattice=1, stream=stream.cuda_stream)

    def tri_inc(i):
        tri.apply_strain(i * WORKLOAD["eps_inc"])
        tri.step(nst)
    out["triangular_2048"] = line(tri, timed(tri, tri_inc), "2048x2048 image, triangular packing",
                                  "k_strip2d (triangular packing: site grid, three forward slots)")
    tri.close()

    sq = lsm.Specimen.from_image(img, k, e, m, dt=WORKLOAD["dt"], damping=WORKLOAD["damping"],
                                 precision=args.precision, stream=stream.cuda_stream)
    sq.apply_strain(WORKLOAD["eps_inc"])
    sq.set_strain_rate(WORKLOAD["eps_inc"] / (nst * WORKLOAD["dt"]))
    out["strain_rate_2048"] = line(sq, timed(sq, lambda i: sq.step(nst)),
                                   "2048x2048 composite, grips at a constant strain rate",
                                   KERNEL.get(args.precision, "k_tile2d") + ", rate-loading instance")
    sq.fields()  # first call allocates the field buffers
    sq.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(3, min(args.steps, 20))
    a.record(stream)
    for _ in range(reps):
        sq.fields()
    b.record(stream)
    stream.synchronize()
    ms = a.elapsed_time(b) / reps
    out["fields_2048"] = {"value": sq.n / (ms * 1e-3), "unit": "particles/s", "ms_per_call": ms,
                          "particles": sq.n, "note": "lsm_fields: per-particle virial stress and Lagrangian "
                          "strain, including the device-to-host copy of both fields (2 x 3 x n doubles)"}
    sq.close()
    return {"workload": "next_rows_2048", "precision": args.precision, "steps": args.steps,
            "warmup": args.warmup, **out}


def _config_2d(n, m, dim, precision, world):
    """The bench line's config for the 2048 x 2048 workload (shared by the
    library arm and the oracle arm)."""
    return {"workload": WORKLOAD["name"], "image": "%dx%d" % (WORKLOAD["nx"], WORKLOAD["ny"]),
            "particles": n, "springs": m, "time_steps_per_bench_step": WORKLOAD["steps_per_increment"],
            "dt": WORKLOAD["dt"], "damping": WORKLOAD["damping"], "precision": precision,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2 (%.0f MB of state and springs per time step)"
                  % (algorithmic_bytes(n, m, dim) / 1e6)}


def run_oracle_sample(budget_s=12.0, threads=1, foam=False):
    """The FP64 CPU oracle on the same workload (the 2048 x 2048 composite, or
    with foam=True the 256^3 foam): one strain increment, then as many time
    steps as fit in about budget_s seconds, on `threads` host threads (the
    oracle's threaded spring pass gives the same bits)."""
    import oracle
    oracle.build_oracle()
    if foam:
        from gen.images import foam_volume, one_phase_materials
        img = foam_volume(256, 4.0, 0.35, seed=2)
        k, e, m = one_phase_materials(1.0, 0.04)
        o = oracle.Oracle.from_image(img, k, e, m, dt=0.01, damping=0.1, grip_mode=1)
        eps, what = -1e-3, "256^3 foam"
    else:
        img = inclusion_image(WORKLOAD["nx"], WORKLOAD["ny"], *WORKLOAD["r"], WORKLOAD["frac"], WORKLOAD["seed"])
        k, e, m = two_phase_materials()
        o = oracle.Oracle.from_image(img, k, e, m, dt=WORKLOAD["dt"], damping=WORKLOAD["damping"])
        eps, what = WORKLOAD["eps_inc"], "2048x2048"
    used = o.set_threads(threads)
    o.apply_strain(eps)
    t0 = time.perf_counter()
    o.step(1)
    one = time.perf_counter() - t0
    nsteps = max(1, int(budget_s / max(one, 1e-6)))
    t0 = time.perf_counter()
    o.step(nsteps)
    dt = time.perf_counter() - t0
    return {"value": o.m * nsteps / dt, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": "%d time steps of the full %s workload after one %g strain increment "
                      "(plain C FP64 oracle, %d host thread%s)" % (nsteps, what, eps, used, "" if used == 1 else "s"),
            "seconds": dt, "steps": nsteps, "n": o.n, "m": o.m}


def cpu_baseline(foam=False):
    """The oracle on all host cores (threaded spring pass), with the
    single-threaded figure beside it."""
    cores = os.cpu_count() or 1
    out = run_oracle_sample(budget_s=15.0, threads=cores, foam=foam)
    one = run_oracle_sample(budget_s=10.0, threads=1, foam=foam)
    for q in (out, one):
        q.pop("n")
        q.pop("m")
    out["single_thread"] = {"value": one["value"], "cores": 1, "sample": one["sample"]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lsm", choices=["lsm", "reference"])
    ap.add_argument("--precision", default="df64", choices=["exact64", "fast64", "f32", "df64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--workload", default="2d_2048", choices=["2d_2048", "batch512", "foam256", "next_rows"])
    ap.add_argument("--no-curves", action="store_true")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.gpus != world:
        # one process per GPU: --gpus N is launched as N torchrun ranks
        print("bench.py: --gpus %d but WORLD_SIZE=%d; launch N>1 under torchrun with --nproc-per-node N"
              % (args.gpus, world), file=sys.stderr)
        return 2
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        if rank != 0:
            return 0
        base = run_oracle_sample(budget_s=max(5.0, min(120.0, 2.0 * args.steps)), threads=os.cpu_count() or 1)
        out = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT,
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": 1e3 * base["seconds"] / base["steps"] * WORKLOAD["steps_per_increment"],
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic (seeded two-phase inclusion image)",
               "config": _config_2d(base.pop("n"), base.pop("m"), 2, "f64", world),
               "cpu_baseline": base,
               "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return 0

    if world > 1:
        import torch
        import torch.distributed as td
        if torch.cuda.is_available():
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        td.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if args.workload == "batch512":
        res = run_batch512(args, rank, world)
        if rank == 0:
            print(json.dumps(res))
        if world > 1:
            import torch.distributed as td
            td.destroy_process_group()
        return 0
    if args.workload == "next_rows":
        if rank == 0:
            print(json.dumps(run_next_rows(args)))
        if world > 1:
            import torch.distributed as td
            td.destroy_process_group()
        return 0
    if args.workload == "foam256":
        if rank == 0:
            out = run_foam256(args)
            if world == 1 and not args.no_cpu_baseline:
                out["cpu_baseline"] = cpu_baseline(foam=True)
            print(json.dumps(out))
        if world > 1:
            import torch.distributed as td
            td.destroy_process_group()
        return 0
    out = run_gpu(args, rank, world)
    if rank == 0 and world == 1 and not args.no_curves:
        out["curves"] = run_curves_subset(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
    if world > 1:
        import torch.distributed as td
        td.barrier()
        td.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
