#!/usr/bin/env python
"""Newton sweeps per second of the local-Newton 3DGS hot path on one B300.

A step is one sweep (Sec. 4.2 group order, Sec. 4.3 secondary targets): for
each of the five attribute groups, render the primary view at full resolution
and its three KNN secondaries at half resolution, accumulate the group's
gradient/Hessian blocks, solve and apply.  The primary cycles through the
cameras.  Default workload ("scene"): 1M Gaussians spread to radius 50, SH
degree 3, 200 cameras 1600x1040 on a smooth trajectory; synthetic inputs,
targets rendered from the ground-truth scene, training starts from a copy
with perturbed means.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gs2|reference]
                    [--workload scene|object|tiny] [--no-cpu-baseline]

Prints one JSON line on rank 0.  --impl reference times the FP64 CPU oracle
(the project's reference implementation of the method) on bounded samples of
the same workload.  Multi-GPU (torchrun) runs independent replicas, one per
GPU, each with its own scene seed; the path has no cross-GPU exchange.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2501_13975_b300 import synth  # noqa: E402

GROUP_NAMES = ("position", "rotation", "scaling", "opacity", "colour")
# FP32 operations of the accumulation per evaluated (pixel, Gaussian) pair
# (a fused multiply-add counts 2): 46 common (falloff and alpha 14, T_k 2,
# weight 1, colour-behind terms 6, e.a 5, h.a^2 8, C_back update 10) + the
# group's payload + its P warp-sum adds.  The geometric payloads are moments
# of the per-pixel weights over monomials of u = Sigma^-1 d: position 132 + 48
# (u 6, monomials 12, weights 3, W1 moments 24, W2 moments 29, colour-path
# weights 15 and moments 30, colour 13), rotation / scaling 43 + 13 (u 6,
# monomials 8, weights 3, W1 moments 10, W2 moments 16), opacity 3 + 2,
# colour 9 + 6
EVAL_FLOPS = (226, 102, 102, 51, 61)
# FP32 peak: 148 SMs x 128 FP32 lanes x 2 FLOP per FMA x 2.032 GHz (maximum SM clock)
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12
PAYLOAD_FLOATS = (48, 13, 13, 2, 6)     # image-space accumulator floats per Gaussian and view
RECORD_BYTES = 40                        # per (tile, Gaussian) pair: id (4) + pi, conic, sigma, c~ (36)
PIXEL_BYTES = 32                         # per pixel: e, h (24) + T_final, last (8)

WORKLOADS = {
    "scene": dict(desc="1M Gaussians spread log-uniformly to radius 50, SH degree 3, 200 cameras 1600x1040 on a "
                       "smooth trajectory; 1 primary (full res) + 3 KNN secondaries (half res) x 5 groups per sweep",
                  n=1_000_000, cams=200, width=1600, height=1040, sh=3, max_pairs=48_000_000),
    "object": dict(desc="100k Gaussians on a unit-sphere shell, SH degree 3, 100 cameras 800x800 on a hemisphere; "
                        "1 primary + 3 KNN secondaries x 5 groups per sweep",
                   n=100_000, cams=100, width=800, height=800, sh=3, max_pairs=24_000_000),
    "tiny": dict(desc="1,000 Gaussians in [-1,1]^3, SH degree 0, 4 cameras 128x128 on a ring",
                 n=1000, cams=4, width=128, height=128, sh=0, max_pairs=1_000_000),
}


def make_workload(name, seed_offset=0):
    w = WORKLOADS[name]
    if name == "scene":
        gt = synth.spread_scene(seed=6 + seed_offset)
        cams = synth.trajectory_cameras(seed=7 + seed_offset)
    elif name == "object":
        gt = synth.object_scene(seed=3 + seed_offset)
        cams = synth.hemisphere_cameras()
    else:
        gt = synth.tiny_scene(seed=1 + seed_offset)
        cams = synth.ring_cameras(4, 128)
    train = synth.perturbed(gt, seed=4 + seed_offset, sd=0.02)
    return w, gt, train, cams


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU arm

def max_over_ranks(values, device):
    """Element-wise maximum of per-rank timings over the process group (the
    slowest replica sets the job's time); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_2501_13975_b300 import gs2

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w, gt_host, train_host, cams = make_workload(args.workload, seed_offset=rank)
    if args.cams:
        cams = cams[: args.cams]
    ncam = len(cams)
    W, H = w["width"], w["height"]
    ctx = gs2.Context(w["n"], W, H, w["sh"], w["max_pairs"], dict(precision=args.precision))
    stream = torch.cuda.current_stream()

    # targets: ground-truth renders of every camera (resident in HBM)
    gt = gs2.DeviceScene.from_host(gt_host)
    targets = []
    proj = ctx.proj_buffer(w["n"])
    for c in cams:
        ctx.project(gt, c, proj)
        img, _ = ctx.raster_fwd(gt, c, proj)
        targets.append(img.clone())
    del gt
    torch.cuda.synchronize()
    ctx.check()

    scene = gs2.DeviceScene.from_host(train_host)
    sphere = ctx.bounding_sphere(scene).cpu().numpy()
    centres = np.stack([c.center() for c in cams]).astype(np.float32)
    knn = gs2.camera_knn(centres, sphere, ctx.config["knn_k"])
    losses = torch.zeros(10, dtype=torch.float64, device=dev)
    nfail = torch.zeros(1, dtype=torch.int32, device=dev)
    tuning = ctx.autotune(scene, cams, targets, knn, 0, reps=2) if not args.no_autotune else ctx.tuning()
    if args.accum_px:
        ctx.set_tuning(accum_px=args.accum_px)
        tuning = dict(tuning, accum_px=args.accum_px)
    if args.accum_split >= 0:
        ctx.set_tuning(accum_split=args.accum_split)
        tuning = dict(tuning, accum_split=args.accum_split)

    # the timed sweeps: through a one-scene gs2_batch captured as a CUDA graph
    # per sweep (re-captured and updated in place: no priming, any primary
    # order), or eagerly through the context (--graph 0)
    batch = prep = None
    if args.graph:
        batch = gs2.Batch([dict(max_gaussians=w["n"], max_width=W, max_height=H, max_sh_degree=w["sh"],
                                max_pairs=w["max_pairs"])], dict(precision=args.precision))
        batch.set_tuning(0, tuning["sort_blocks"], tuning["sort_rows"], tuning["view_lanes"], tuning["accum_px"],
                         tuning["accum_split"])
        prep = batch.prepare([scene], [cams], [targets], [knn])

    def sweep(i, tg=None):
        if batch is not None:
            if tg is not None:
                batch.set_targets(prep, 0, tg)
            batch.sweep(prep, [i % ncam], losses, nfail, use_graph=args.graph)
        else:
            ctx.sweep(scene, cams, targets if tg is None else tg, knn, i % ncam, losses, nfail)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def check():
        ctx.check()
        if batch is not None:
            batch.check()

    for i in range(args.warmup):
        sweep(i)
    torch.cuda.synchronize()
    check()

    # ---------------- device-resident timed region (the views of each group concurrent)
    clocks = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    l0 = gs2.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(args.steps):
        sweep(args.warmup + i)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = gs2.launch_count() - l0
    clk = clocks.stop()
    barrier()
    ms = ev0.elapsed_time(ev1)
    check()

    # ---------------- roofline pass (untimed): the same sweeps with the views one
    # after another, so that each accumulation launch's CUDA-event duration is
    # its own and not shared with a concurrent view
    lanes_on = ctx.tuning()["view_lanes"]
    ctx.set_tuning(view_lanes=0)
    ctx.profile(True)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for i in range(args.steps):
        ctx.sweep(scene, cams, targets, knn, (args.warmup + args.steps + i) % ncam, losses, nfail)
    p1.record(stream)
    torch.cuda.synchronize()
    ms_serial = p0.elapsed_time(p1)
    prof = ctx.profile_read()
    ctx.profile(False)
    ctx.set_tuning(view_lanes=lanes_on)
    ctx.check()

    # ---------------- end to end through the public API with host buffers: the
    # targets live in pinned host memory (HostTargets); each sweep's views are
    # uploaded on a copy stream, the next sweep's while the current one runs.
    # Every timed step's upload happens inside the timed region: none is
    # prefetched before it starts or after it ends.
    ht = gs2.HostTargets([t.cpu() for t in targets], knn)
    host_losses = torch.zeros(10, dtype=torch.float64).pin_memory()
    host_nfail = torch.zeros(1, dtype=torch.int32).pin_memory()
    h2d = ht.bytes_for(0)
    d2h = host_losses.numel() * 8 + host_nfail.numel() * 4

    def e2e_step(i, prefetch_next):
        t = i % ncam
        sweep(i, ht.targets(t))
        ht.release(t)
        if prefetch_next:
            ht.prefetch((i + 1) % ncam)
        host_losses.copy_(losses, non_blocking=True)
        host_nfail.copy_(nfail, non_blocking=True)

    for i in range(args.warmup):
        e2e_step(1000 + i, i + 1 < args.warmup)
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        e2e_step(1000 + args.warmup + i, i + 1 < args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = e0.elapsed_time(e1)
    check()

    # the extra timings below use the device-resident targets again
    if batch is not None:
        batch.set_targets(prep, 0, targets)
    # ---------------- the plain FP32 path on the same workload, timed the same
    # way (device-resident, one graph per sweep), beside the precision form
    fp32_path = None
    if args.precision == 1 and not args.no_fp32_path:
        if batch is not None:
            batch.set_config(0, precision=0)
        ctx.set_config(precision=0)
        for i in range(2):
            sweep(2000 + i)
        torch.cuda.synchronize()
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for i in range(args.steps):
            sweep(2002 + i)
        f1.record(stream)
        torch.cuda.synchronize()
        barrier()
        check()
        fms = f0.elapsed_time(f1) / args.steps
        fp32_path = {"sweeps_per_s": round(1000.0 / fms, 4), "ms_per_sweep": round(fms, 3),
                     "what": "the same sweeps with precision 0 (FP32 accumulation, FP32 solves only)"}
        if batch is not None:
            batch.set_config(0, precision=args.precision)
        ctx.set_config(precision=args.precision)

    # ---------------- deterministic mode (identical bytes on every run: per-entry
    # partials, fixed-order sums, views one after another), timed the same way
    det_path = None
    if not args.no_det_path:
        if batch is not None:
            batch.set_config(0, deterministic=1)
        ctx.set_config(deterministic=1)
        for i in range(2):
            sweep(3000 + i)
        torch.cuda.synchronize()
        barrier()
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        nd = max(1, min(args.steps, 5))
        d0.record(stream)
        for i in range(nd):
            sweep(3002 + i)
        d1.record(stream)
        torch.cuda.synchronize()
        barrier()
        check()
        dms = d0.elapsed_time(d1) / nd
        det_path = {"sweeps_per_s": round(1000.0 / dms, 4), "ms_per_sweep": round(dms, 3), "sweeps": nd,
                    "what": "deterministic = 1 with the headline's precision (bit-identical blocks and parameters)"}
        if batch is not None:
            batch.set_config(0, deterministic=0)
        ctx.set_config(deterministic=0)

    if world > 1:
        ms, ms_e2e = max_over_ranks([ms, ms_e2e], dev)

    # ---------------- the single-render variant (Jacobi over groups), timed
    # beside the paper's in-series sweep on the same workload: a different
    # method, reported apart from `value`
    jacobi = None
    if not args.no_variants:
        cj = gs2.Context(w["n"], W, H, w["sh"], w["max_pairs"], dict(precision=args.precision, group_jacobi=1))
        cj.set_tuning(**{k: tuning[k] for k in ("sort_blocks", "sort_rows", "view_lanes", "accum_px", "accum_split")})
        sj = scene.clone()
        for i in range(2):
            cj.sweep(sj, cams, targets, knn, i % ncam)
        torch.cuda.synchronize()
        j0 = torch.cuda.Event(enable_timing=True)
        j1 = torch.cuda.Event(enable_timing=True)
        j0.record(stream)
        for i in range(args.steps):
            cj.sweep(sj, cams, targets, knn, (args.warmup + i) % ncam)
        j1.record(stream)
        torch.cuda.synchronize()
        cj.check()
        jms = j0.elapsed_time(j1) / args.steps
        jacobi = {"sweeps_per_s": round(1000.0 / jms, 3), "ms_per_sweep": round(jms, 3), "launch": "eager",
                  "method": "every view rendered once per sweep; all groups solved at that state (group_jacobi)"}
        cj.close()
        del sj

    # ---------------- roofline of the accumulation kernel: bound by its per-pair
    # arithmetic (ALU), not HBM; the HBM figure with algorithmic bytes beside it
    peak, peak_kind = load_peaks()
    accum_ms = float(prof["accum_ms"].sum())
    n_acc = int(prof["accum_launches"].sum())
    alg_bytes = 0.0
    for g in range(5):
        alg_bytes += (PIXEL_BYTES * float(prof["pixels"][g]) + RECORD_BYTES * float(prof["listed"][g])
                      + 8.0 * PAYLOAD_FLOATS[g] * float(prof["visible"][g]))
    flops = sum(EVAL_FLOPS[g] * float(prof["evaluations"][g]) for g in range(5))
    hbm_gbs = alg_bytes / (accum_ms * 1e-3) / 1e9 if accum_ms > 0 else 0.0
    tflops = flops / (accum_ms * 1e-3) / 1e12 if accum_ms > 0 else 0.0
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "accum_traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            td = json.load(f)
        if td.get("workload") == args.workload and td.get("kernel_rev") == KERNEL_REV:
            traffic = td.get("bytes_per_launch")
    roofline = {"kernel": "k_accum (all groups)", "bound": "alu", "achieved": round(tflops, 3),
                "peak": round(FP32_PEAK_TFLOPS, 2), "unit": "TFLOP/s", "frac": round(tflops / FP32_PEAK_TFLOPS, 4),
                "traffic": traffic,
                "peak_source": "148 SMs x 128 FP32 lanes x 2 x 2.032 GHz",
                "flops_per_launch": round(flops / max(n_acc, 1)),
                "evaluations_per_sweep": int(prof["evaluations"].sum()) // max(args.steps, 1),
                "hbm": {"achieved": round(hbm_gbs, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(hbm_gbs / peak, 4), "peak_source": peak_kind,
                        "algorithmic_bytes_per_launch": round(alg_bytes / max(n_acc, 1))},
                "launches": n_acc,
                "avg_launch_ms": round(accum_ms / max(n_acc, 1), 4),
                "share_of_step": round(accum_ms / ms_serial, 4) if ms_serial > 0 else None,
                "measured_in": "untimed pass with the views of a group one after another "
                               f"({ms_serial / args.steps:.2f} ms/sweep; the timed sweeps run them concurrently)",
                "pairs_per_sweep": int(prof["pairs"].sum()) // max(args.steps, 1),
                "listed_pairs_per_sweep": int(prof["listed"].sum()) // max(args.steps, 1),
                "visible_per_binning": int(prof["visible"].sum()) // max(int(prof["binnings"].sum()), 1)}
    # ---------------- the other stages, reported separately (same serial pass):
    # algorithmic bytes per sweep against the measured HBM peak
    binn = prof["binnings"].astype(np.float64)
    pairs = float(prof["pairs"].sum())       # sorted: one per tile of each support rectangle
    listed = float(prof["listed"].sum())     # in the tile lists: tiles the support ellipse reaches
    visible = float(prof["visible"].sum())
    pixels = float(prof["pixels"].sum())
    depth_sorts = float(binn[0] + binn[1])   # the position and rotation passes sort by depth
    stage_bytes = {
        # per emitted pair: emit 8 B, first tile radix pass 4 B histogram read + 8 B read; per listed
        # pair (the first pass drops the others): its 8 B write, the second pass 20 B, ranges 4 B;
        # four depth radix passes of 20 B per Gaussian; the tiles-touched scan 16 B per Gaussian
        # (order and touched read, tsort and offsets written); the support ellipse's parameters
        # read by the emission, 24 B per visible one
        "binning": pairs * (8 + 12) + listed * (8 + 20 + 4) + depth_sorts * w["n"] * 4 * 20
                   + float(binn.sum()) * w["n"] * 16 + visible * 24,
        # per pixel 12 B image + 8 B state written; per listed pair 4 B id + 48 B staged record
        "compositing": pixels * 20 + listed * 52,
        # per pixel c, target read (24 B), e, h written (24 B)
        "loss": pixels * 48,
    }
    stages = {}
    for k, b in stage_bytes.items():
        t_ms = float(prof["stage_ms"][k])
        gbs = b / (t_ms * 1e-3) / 1e9 if t_ms > 0 else 0.0
        stages[k] = {"ms_per_sweep": round(t_ms / max(args.steps, 1), 3), "launch_groups": prof["stage_count"][k],
                     "algorithmic_bytes_per_sweep": round(b / max(args.steps, 1)),
                     "achieved_gbs": round(gbs, 1), "hbm_frac": round(gbs / peak, 4),
                     "share_of_step": round(t_ms / ms_serial, 4) if ms_serial > 0 else None}
    value = world * args.steps / (ms * 1e-3)
    result = {
        "metric": "Newton sweeps/s (1 primary + 3 secondaries, 5 attribute groups)",
        "value": round(value, 4), "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == 0 else "f32+f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {w['desc']}", "gaussians": w["n"], "cameras": ncam,
                   "width": W, "height": H, "sh_degree": w["sh"], "knn_k": ctx.config["knn_k"],
                   "downsample": ctx.config["downsample"], "lambda_ssim": ctx.config["lambda_ssim"],
                   "precision": "fp32" if args.precision == 0 else "mixed (FP64 accumulation, FP64 re-solve if cond > 1e6)",
                   "l2": "inputs larger than L2 (scene parameters and targets exceed 126 MB)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "e2e": {"value": round(world * args.steps / (ms_e2e * 1e-3), 4), "unit": "sweeps/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "roofline": roofline,
        "stages": stages,
        "jacobi_groups": jacobi,
        "fp32_path": fp32_path,
        "deterministic_path": det_path,
        "gpu_launches": int(launches),
        "tuning": tuning,
        "launch": "one CUDA graph per sweep (captured, updated in place)" if args.graph else "eager",
        "clocks": clk,
        "accumulate_ms_by_group": {GROUP_NAMES[g]: round(float(prof["accum_ms"][g]) / max(args.steps, 1), 3)
                                   for g in range(5)},
        "n_failed_total": int(nfail.item()),
        "primary_loss_last": [round(float(x), 6) for x in host_losses[:2]],
    }
    return result, (w, train_host, cams)


# ----------------------------------------------------------------------------- batched scenes

def run_batched(args):
    """Batched form: 16 independent scenes (Gaussian counts log-uniform in
    [20k, 500k], 16-128 views, 512x512 to 1024x768, SH degree 3, shells and
    spread scenes alternating; seed 8) swept together, one sweep per scene per
    batched sweep (primary = sweep index mod views).  Per scene the kernel
    tuning is chosen by gs2_autotune first.  Timed per batched sweep with CUDA
    events: the scenes one after another on one stream, the scenes forked
    onto their own streams, the same captured as one CUDA graph per batched
    sweep (updated in place), and graphs kept per scene and primary (replayed
    when a primary comes round again); scenes/s = scenes x sweeps / time."""
    import ctypes as C

    import torch
    from paper_2501_13975_b300 import gs2

    torch.cuda.set_device(0)
    work = synth.batched_workload(seed=8)
    if args.batched_only:   # a subset of the 16 scenes (profiling captures)
        work = [work[int(i)] for i in args.batched_only.split(",")]
    sizes = [dict(max_gaussians=w["n"], max_width=w["width"], max_height=w["height"], max_sh_degree=3,
                  max_pairs=96 * w["n"]) for w in work]
    batch = gs2.Batch(sizes)
    stream = torch.cuda.current_stream()
    starts, scenes, targets, knns = [], [], [], []
    for w in work:
        tmp = gs2.Context(w["n"], w["width"], w["height"], 3, 96 * w["n"])
        gt = gs2.DeviceScene.from_host(w["gt"])
        proj = tmp.proj_buffer(w["n"])
        tg = []
        for c in w["cams"]:
            tmp.project(gt, c, proj)
            img, _ = tmp.raster_fwd(gt, c, proj)
            tg.append(img.clone())
        ds = gs2.DeviceScene.from_host(w["train"])
        sphere = tmp.bounding_sphere(ds).cpu().numpy()
        centres = np.stack([c.center() for c in w["cams"]]).astype(np.float32)
        knns.append(gs2.camera_knn(centres, sphere, 3))
        targets.append(tg)
        scenes.append(ds)
        starts.append(ds.clone())
        tmp.close()
    torch.cuda.synchronize()
    tuning = []
    t0 = time.perf_counter()
    if not args.no_autotune:
        for i, w in enumerate(work):
            tuning.append(batch.autotune(i, scenes[i], w["cams"], targets[i], knns[i], 0, reps=2))
    if args.accum_split >= 0:
        for i, w in enumerate(work):
            cur = tuning[i] if tuning else batch.tuning(i)
            batch.set_tuning(i, cur["sort_blocks"], cur["sort_rows"], cur["view_lanes"], cur["accum_px"],
                             args.accum_split)
    t_tune = time.perf_counter() - t0
    prep = batch.prepare(scenes, [w["cams"] for w in work], targets, knns)
    views = [w["views"] for w in work]

    def restore():
        for ds, st0 in zip(scenes, starts):
            for name in ("mean", "quat", "scale", "opacity", "sh"):
                getattr(ds, name).copy_(getattr(st0, name))

    def timed(mode, steps, warmup):
        if mode == "graph_kept":
            # steady state of a training run: every (scene, primary) graph captured
            # once first (the graphs reference the scene buffers, so restoring the
            # start afterwards keeps them valid)
            restore()
            for i in range(max(views)):
                batch.sweep(prep, [i % v for v in views], use_graph=2)
            torch.cuda.synchronize()
        restore()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(warmup + steps):
            t = [i % v for v in views]
            if i >= warmup:
                ev[i - warmup][0].record(stream)
            if mode == "sequential":
                for s in range(len(work)):
                    gs2._lib.gs2_sweep(batch.ctx_handle(s), C.byref(prep["scenes"][s]), prep["cams"][s],
                                       len(work[s]["cams"]), prep["tgts"][s], prep["knn"][s], t[s], None, None,
                                       gs2._stream(None))
            else:
                batch.sweep(prep, t, use_graph={"streams": 0, "graph": 1, "graph_kept": 2}[mode])
            if i >= warmup:
                ev[i - warmup][1].record(stream)
        torch.cuda.synchronize()
        batch.check()
        ms = np.array([a.elapsed_time(b) for a, b in ev])
        return {"scenes_per_s": round(len(work) * steps / (ms.sum() * 1e-3), 3),
                "ms_per_batched_sweep": {"p50": round(float(np.percentile(ms, 50)), 3),
                                         "p99": round(float(np.percentile(ms, 99)), 3),
                                         "mean": round(float(ms.mean()), 3)}}

    res = {}
    l0 = gs2.launch_count()
    for mode in ("sequential", "streams", "graph", "graph_kept"):
        res[mode] = timed(mode, args.steps, args.warmup)
    launches = gs2.launch_count() - l0
    head = max((res["graph"], res["graph_kept"]), key=lambda r: r["scenes_per_s"])
    return {
        "metric": f"scenes/s (batched sweeps, {len(work)} independent scenes)", "value": head["scenes_per_s"],
        "unit": "scenes/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": head["ms_per_batched_sweep"]["mean"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched: 16 scenes, N log-uniform [20k, 500k], 16-128 views, 512x512..1024x768, "
                               "SH3, shells and spread scenes alternating (seed 8)",
                   "subset": args.batched_only or None,
                   "gaussians_total": int(sum(w["n"] for w in work)),
                   "scenes": [{k: w[k] for k in ("kind", "n", "views", "width", "height")} for w in work],
                   "sweep_restart": "every mode starts from the training start"},
        "modes": res,
        "graph": batch.stats(),
        "autotune": {"seconds": round(t_tune, 2), "choices": tuning},
        "gpu_launches": int(launches),
    }


# ----------------------------------------------------------------------------- method variants

def method_variants(args):
    """The paper's two ablations and the Gauss-Newton variant on the object
    workload, with the same kernels: 30 sweeps (primaries in a seeded
    permutation, seed 5) from the workload's start for each of
      paper        K = 3 secondaries, order position, rotation, scaling, opacity, colour
      K=0, K=8     secondary targets per primary (Sec. 5, trade-off of secondary targets)
      colour-first order colour, opacity, scaling, rotation, position (Sec. 5, optimisation order)
      gauss-newton Gauss-Newton blocks: the e d2c/dy2 terms left out (Sec. 6)
      jacobi-groups every view rendered once per sweep, all groups solved at that
                   state and applied together (the single-render variant)
    PSNR over all 100 views after every sweep (outside the timed work) and the
    sweeps' device time (CUDA events)."""
    import torch
    from paper_2501_13975_b300 import gs2

    torch.cuda.set_device(0)
    w, gt_host, start_host, cams = make_workload("object")
    if args.variants_n or args.variants_sd:
        # the same shell with fewer Gaussians (less overlap between them) and/or
        # a start closer to the target (smaller perturbation of the means)
        if args.variants_n:
            w = dict(w, n=args.variants_n)
            gt_host = synth.object_scene(seed=3, n=args.variants_n)
        start_host = synth.perturbed(gt_host, seed=4, sd=args.variants_sd or 0.02)
    # mean overlap of the shell: Gaussians covering a point of it, taking each
    # footprint as a disc of radius 2 s (s = its mean scale)
    s_mean = np.exp(np.log(gt_host.scale.astype(np.float64)).mean(axis=0))
    r_mean = np.linalg.norm(gt_host.mean.astype(np.float64), axis=0).mean()
    overlap = float(np.sum(np.pi * (2.0 * s_mean) ** 2) / (4.0 * np.pi * r_mean ** 2))
    ncam = len(cams)
    W, H = w["width"], w["height"]
    order = np.random.Generator(np.random.PCG64(5)).permutation(ncam)
    variants = [("paper", {}), ("K=0", dict(knn_k=0)), ("K=8", dict(knn_k=8)),
                ("colour-first", dict(group_order=(4, 3, 2, 1, 0))), ("gauss-newton", dict(gauss_newton=1)),
                ("jacobi-groups", dict(group_jacobi=1))]
    if args.variants_only:
        variants = [v for v in variants if v[0] in args.variants_only.split(",")]
    extra = {}
    for kv in filter(None, args.variants_cfg.split(",")):
        k, v = kv.split("=")
        extra[k] = float(v) if "." in v or "e" in v else int(v)
    variants = [(name, dict(extra, **cfg)) for name, cfg in variants]
    sweeps = 30
    out = {}
    for name, cfg in variants:
        ctx = gs2.Context(w["n"], W, H, w["sh"], w["max_pairs"], cfg)
        gt = gs2.DeviceScene.from_host(gt_host)
        proj = ctx.proj_buffer(w["n"])
        targets = []
        for c in cams:
            ctx.project(gt, c, proj)
            img, _ = ctx.raster_fwd(gt, c, proj)
            targets.append(img.clone())
        del gt
        scene = gs2.DeviceScene.from_host(start_host)
        sphere = ctx.bounding_sphere(scene).cpu().numpy()
        centres = np.stack([c.center() for c in cams]).astype(np.float32)
        knn = gs2.camera_knn(centres, sphere, ctx.config["knn_k"])
        evl = torch.zeros((ncam, 2), dtype=torch.float64, device="cuda")
        nfail = torch.zeros(1, dtype=torch.int32, device="cuda")

        def psnr():
            evl.zero_()
            for v, c in enumerate(cams):
                ctx.project(scene, c, proj)
                img, _ = ctx.raster_fwd(scene, c, proj)
                ctx.loss_derivs(img, targets[v], loss=evl[v])
            mse = 2.0 * evl[:, 0].cpu().numpy()
            return float(np.mean(10.0 * np.log10(1.0 / np.maximum(mse, 1e-30))))

        curve, ms = [psnr()], 0.0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for i in range(sweeps):
            e0.record()
            ctx.sweep(scene, cams, targets, knn, int(order[i % ncam]), None, nfail)
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            curve.append(psnr())
        ctx.check()
        out[name] = {"config": {k: (list(v) if isinstance(v, tuple) else v) for k, v in cfg.items()},
                     "psnr_start": round(curve[0], 4), "psnr_after_1": round(curve[1], 4),
                     "psnr_after_30": round(curve[-1], 4), "best_psnr": round(max(curve), 4),
                     "ms_per_sweep": round(ms / sweeps, 3), "failed_solves": int(nfail.item()),
                     "psnr_curve": [round(x, 3) for x in curve]}
        ctx.close()
    return {"metric": "PSNR over all views after 30 sweeps, per method variant (object workload)",
            "value": out["paper"]["psnr_after_30"], "unit": "dB", "higher_is_better": True,
            "config": {"workload": f"object: {w['n']} Gaussians on a unit-sphere shell, SH degree 3, 100 cameras "
                                   f"800x800 on a hemisphere; start: means perturbed N(0, {args.variants_sd or 0.02}^2)",
                       "gaussians": w["n"], "shell_overlap": round(overlap, 1),
                       "primaries": "seeded permutation (seed 5)"},
            "data": "synthetic", "dtype": "f32", "variants": out}


# ----------------------------------------------------------------------------- first-order baseline

def gd_baseline(args):
    """First-order baseline on the same kernels (gd_lr): every group steps by
    -lr g instead of its damped Newton step, inside the same trust radii and
    bounds; the rest of the sweep (views, secondary targets, group order) is
    the paper's.  Object workload, primaries in a seeded permutation (seed 5),
    from the workload's start.  Learning rates: lr_g = eta / median |diag H_g|
    over the Gaussians with a block, from the blocks of the first primary's
    view at the start (a one-off scale calibration per group), for eta in
    {1e-4, 1e-3, 0.01, 0.1, 1}.  100 sweeps each, PSNR over all views after sweeps 1, 3,
    10, 30 and 100, against the Newton sweep's PSNR after sweep 1 (the paper's
    claim: one Newton iteration does as well as 100 or more gradient ones)."""
    import torch
    from paper_2501_13975_b300 import gs2

    torch.cuda.set_device(0)
    w, gt_host, start_host, cams = make_workload("object")
    ncam = len(cams)
    W, H = w["width"], w["height"]
    order = np.random.Generator(np.random.PCG64(5)).permutation(ncam)
    ctx = gs2.Context(w["n"], W, H, w["sh"], w["max_pairs"])
    gt = gs2.DeviceScene.from_host(gt_host)
    proj = ctx.proj_buffer(w["n"])
    targets = []
    for c in cams:
        ctx.project(gt, c, proj)
        img, _ = ctx.raster_fwd(gt, c, proj)
        targets.append(img.clone())
    del gt
    start = gs2.DeviceScene.from_host(start_host)
    sphere = ctx.bounding_sphere(start).cpu().numpy()
    knn = gs2.camera_knn(np.stack([c.center() for c in cams]).astype(np.float32), sphere, ctx.config["knn_k"])
    n, S = w["n"], (w["sh"] + 1) ** 2

    # scale calibration: median |diag H| per group on the first primary's view
    cam0 = cams[int(order[0])]
    p0 = ctx.project(start, cam0)
    img0, rs0 = ctx.raster_fwd(start, cam0, p0)
    base = []
    for g in gs2.GROUPS:
        b = ctx.blocks_buffer(g, n, w["sh"], 1)
        ctx.accum(g, start, cam0, cam0, p0, rs0, img0, targets[int(order[0])], 0, b)
        bb = b.cpu().numpy()
        if g in (gs2.POS, gs2.SCALE):
            d = np.abs(bb[3 * n:9 * n].reshape(6, n)[[0, 3, 5]]).mean(axis=0)
        elif g in (gs2.ROT, gs2.OPACITY):
            d = np.abs(bb[n:2 * n])
        else:   # colour slot: sum_p w^2 h per channel times |b|^2 (mean over channels)
            sl = bb[: (6 + S) * n].reshape(6 + S, n)
            d = np.abs(sl[3:6]).mean(axis=0) * (sl[6:] ** 2).sum(axis=0) / S
        d = d[d > 0]
        base.append(float(1.0 / np.median(d)) if d.size else 0.0)

    def psnr(scene):
        evl = torch.zeros((ncam, 2), dtype=torch.float64, device="cuda")
        for v, c in enumerate(cams):
            ctx.project(scene, c, proj)
            img, _ = ctx.raster_fwd(scene, c, proj)
            ctx.loss_derivs(img, targets[v], loss=evl[v])
        mse = 2.0 * evl[:, 0].cpu().numpy()
        return float(np.mean(10.0 * np.log10(1.0 / np.maximum(mse, 1e-30))))

    marks = (1, 3, 10, 30, 100)
    ctx.set_config(gd_lr=[0.0] * 5)
    newton = start.clone()
    ctx.sweep(newton, cams, targets, knn, int(order[0]))
    out = {"psnr_start": round(psnr(start), 4), "newton_psnr_after_1": round(psnr(newton), 4),
           "lr_base": [float(f"{b:.4g}") for b in base], "runs": {}}
    for eta in (1e-4, 1e-3, 0.01, 0.1, 1.0):
        ctx.set_config(gd_lr=[eta * b for b in base])
        sc = start.clone()
        curve, ms = {}, 0.0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for i in range(max(marks)):
            e0.record()
            ctx.sweep(sc, cams, targets, knn, int(order[i % ncam]))
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            if i + 1 in marks:
                curve[i + 1] = round(psnr(sc), 4)
        ctx.check()
        out["runs"][f"eta={eta}"] = {"psnr_after": curve, "ms_per_sweep": round(ms / max(marks), 3)}
    best = max(out["runs"].values(), key=lambda r: r["psnr_after"][100])
    return {"metric": "PSNR over all views: 100 gradient sweeps vs 1 Newton sweep (object workload)",
            "value": best["psnr_after"][100], "unit": "dB", "higher_is_better": True,
            "config": {"workload": "object: 100k Gaussians on a unit-sphere shell, SH degree 3, 100 cameras 800x800; "
                                   "start: means perturbed N(0, 0.02^2)", "primaries": "seeded permutation (seed 5)"},
            "data": "synthetic", "dtype": "f32", **out}


# ----------------------------------------------------------------------------- time to PSNR

def time_to_psnr(args):
    """Time to PSNR on the object workload.  The plain FP32 path runs 30
    sweeps (primaries in a seeded permutation, seed 5); the learned paths
    (step-scale network, damping network, both, each with the mixed-precision
    policy; --ttp-paths) then run from the same start until their PSNR over
    all training views reaches the plain path's PSNR after 30 sweeps (at most
    --ttp-max sweeps).  Two starts: the workload's own (means
    perturbed, everything else exact) and the initialised state a training
    run starts from (grey colour, opacity 0.1, jittered scales).  Times are the
    sweeps' device time (CUDA events); PSNR is taken between sweeps, outside
    the timed work.  The network is trained first on records the plain method
    logs on tiny scenes and on smaller shell scenes (other seeds); their
    collection and training times are reported beside it."""
    import torch
    from paper_2501_13975_b300 import gs2, learned

    torch.cuda.set_device(0)
    w, gt_host, spec_host, cams = make_workload("object")
    init_host = synth.initialised(spec_host, seed=9)
    ncam = len(cams)
    W, H = w["width"], w["height"]
    order = np.random.Generator(np.random.PCG64(5)).permutation(ncam)

    # ---- network: records of the plain method, then Adam
    t0 = time.perf_counter()
    tiny, tiny_d = learned.collect_records(range(100, 100 + args.ttp_runs), kind="tiny", damping=True)
    shell, shell_d = learned.collect_records(range(1000, 1000 + args.ttp_shell), kind="shell",
                                             sweeps=args.ttp_shell_sweeps, damping=True)
    torch.cuda.synchronize()
    t_collect = time.perf_counter() - t0
    parts = [r.split(0.1) for r in (tiny, shell)]
    train_sets = [p[0] for p in parts]
    held = [p[1] for p in parts]
    dparts = [r.split(0.1) for r in (tiny_d, shell_d)]
    model = learned.StepModel(seed=20)
    damp = learned.StepModel(seed=22)
    t0 = time.perf_counter()
    model.fit(train_sets, epochs=args.ttp_epochs, batch=16384, objective=args.ttp_objective)
    damp.fit([p[0] for p in dparts], epochs=args.ttp_epochs, batch=16384, objective=args.ttp_damping_objective,
             seed=23)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    held_stats = {}
    for name, hs, hd in zip(("tiny", "shell"), held, [p[1] for p in dparts]):
        pl, cnt = learned.plain_loss(hs)
        nl, _ = model.loss(hs)
        pll, _ = learned.plain_loss(hs, objective="line")
        nll, _ = model.loss(hs, objective="line")
        dpl, dcnt = learned.plain_loss(hd)        # rho = 1 (alpha = 1) against the damping labels
        dnl, _ = damp.loss(hd)
        dwpl, _ = learned.plain_loss(hd, objective="line")   # the same, weighted by the spread of Q
        dwnl, _ = damp.loss(hd, objective="line")
        dl = hd.labels().cpu().numpy()
        dl = dl[dl >= 0]
        held_stats[name] = {"records": cnt, "label_loss_plain": round(pl, 5), "label_loss_network": round(nl, 5),
                            "line_loss_plain": float(f"{pll:.5g}"), "line_loss_network": float(f"{nll:.5g}"),
                            "damping_records": dcnt, "damping_label_loss_plain": round(dpl, 5),
                            "damping_label_loss_network": round(dnl, 5),
                            "damping_weighted_loss_plain": float(f"{dwpl:.5g}"),
                            "damping_weighted_loss_network": float(f"{dwnl:.5g}"),
                            "damping_label_histogram": {f"rho=1e{1.5 * v:.1f}": int(np.sum(
                                np.abs(dl - v) < 1e-4)) for v in np.linspace(0.0, 2.0, 7)}}

    def run(start_host, precision, use_model, max_sweeps, target_psnr=None, learned_trust=None, use_damp=False):
        lt = args.ttp_learned_trust if learned_trust is None else learned_trust
        ctx = gs2.Context(w["n"], W, H, w["sh"], w["max_pairs"], dict(precision=precision, learned_trust=lt))
        gt = gs2.DeviceScene.from_host(gt_host)
        proj = ctx.proj_buffer(w["n"])
        targets = []
        for c in cams:
            ctx.project(gt, c, proj)
            img, _ = ctx.raster_fwd(gt, c, proj)
            targets.append(img.clone())
        del gt
        scene = gs2.DeviceScene.from_host(start_host)
        sphere = ctx.bounding_sphere(scene).cpu().numpy()
        centres = np.stack([c.center() for c in cams]).astype(np.float32)
        knn = gs2.camera_knn(centres, sphere, ctx.config["knn_k"])
        if use_model:
            ctx.set_step_model(model.w)
        if use_damp:
            ctx.set_damping_model(damp.w)
        evl = torch.zeros((ncam, 2), dtype=torch.float64, device="cuda")

        def psnr():
            evl.zero_()
            for v, c in enumerate(cams):
                ctx.project(scene, c, proj)
                img, _ = ctx.raster_fwd(scene, c, proj)
                ctx.loss_derivs(img, targets[v], loss=evl[v])
            mse = 2.0 * evl[:, 0].cpu().numpy()          # L2 = 1/(3|I|) sum 1/2 (c - c^t)^2
            return float(np.mean(10.0 * np.log10(1.0 / np.maximum(mse, 1e-30))))

        curve = [psnr()]
        ms_total = 0.0
        ms_curve = [0.0]
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        reached = None
        for i in range(max_sweeps):
            ev0.record()
            ctx.sweep(scene, cams, targets, knn, int(order[i % ncam]))
            ev1.record()
            torch.cuda.synchronize()
            ms_total += ev0.elapsed_time(ev1)
            ms_curve.append(ms_total)
            curve.append(psnr())
            if target_psnr is not None and reached is None and curve[-1] >= target_psnr:
                reached = i + 1
                if i + 1 >= 30:
                    break
        ctx.check()
        return dict(psnr=curve, ms=ms_curve, reached=reached, sweeps=len(curve) - 1)

    def first_sweep_ms(precision, use_model, reps=5, use_damp=False):
        """Median device time of the first sweep from the workload's start,
        each repetition from a fresh copy of it: the cost of the network's
        inference and of the precision policy on one scene state (the runs
        above move through different states, so their per-sweep times also
        reflect how far each has diverged)."""
        ctx = gs2.Context(w["n"], W, H, w["sh"], w["max_pairs"],
                          dict(precision=precision, learned_trust=args.ttp_learned_trust))
        gt = gs2.DeviceScene.from_host(gt_host)
        proj = ctx.proj_buffer(w["n"])
        targets = []
        for c in cams:
            ctx.project(gt, c, proj)
            img, _ = ctx.raster_fwd(gt, c, proj)
            targets.append(img.clone())
        del gt
        centres = np.stack([c.center() for c in cams]).astype(np.float32)
        sphere = ctx.bounding_sphere(gs2.DeviceScene.from_host(spec_host)).cpu().numpy()
        knn = gs2.camera_knn(centres, sphere, ctx.config["knn_k"])
        if use_model:
            ctx.set_step_model(model.w)
        if use_damp:
            ctx.set_damping_model(damp.w)
        times = []
        for _ in range(reps + 1):
            scene = gs2.DeviceScene.from_host(spec_host)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.sweep(scene, cams, targets, knn, int(order[0]))
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ctx.check()
        return round(float(np.median(times[1:])), 3)

    def med(xs):
        """Median with unreached runs (None) counted as slower than any reached one."""
        v = sorted(float("inf") if x is None else x for x in xs)
        m = v[len(v) // 2] if len(v) % 2 else 0.5 * (v[len(v) // 2 - 1] + v[len(v) // 2])
        return None if m == float("inf") else m

    R = max(1, args.ttp_reps)
    starts = {}
    for sname, host in (("workload", spec_host), ("initialised", init_host)):
        # the trajectories depend on the order of floating-point atomic
        # additions, so every path runs R times: medians, with the spread
        plains = [run(host, 0, False, 30) for _ in range(R)]
        target = float(np.median([p["psnr"][30] for p in plains]))
        t_plain = float(np.median([p["ms"][30] for p in plains])) * 1e-3
        runs = {"plain_fp32": plains}
        # path: (precision, step-scale network, learned_trust, damping network)
        paths = {"learned_mixed": (1, True, None, False), "learned_fp32": (0, True, None, False),
                 "learned_mixed_radii_x2": (1, True, 2.0, False), "damping_mixed": (1, False, None, True),
                 "damping_scale_mixed": (1, True, None, True), "plain_mixed": (1, False, None, False)}
        for name in args.ttp_paths.split(","):
            prec, use, lt, ud = paths[name]
            runs[name] = [run(host, prec, use, max(args.ttp_max, 30), target, lt, ud) for _ in range(R)]
        head_path = "damping_mixed" if "damping_mixed" in runs else "learned_mixed"

        def per_path(rs):
            secs = [r["ms"][r["reached"]] * 1e-3 if r["reached"] is not None else None for r in rs]
            return {"sweeps_to_target": [r["reached"] for r in rs],
                    "median_sweeps_to_target": med([r["reached"] for r in rs]),
                    "seconds_to_target": [None if x is None else round(x, 5) for x in secs],
                    "median_seconds_to_target": None if med(secs) is None else round(med(secs), 5),
                    "psnr_at_30": [round(r["psnr"][min(30, r["sweeps"])], 4) for r in rs],
                    "ms_per_sweep": round(float(np.median([r["ms"][-1] / max(r["sweeps"], 1) for r in rs])), 3)}

        t_lm = med([r["ms"][r["reached"]] * 1e-3 if r["reached"] is not None else None for r in runs[head_path]])
        starts[sname] = {
            "initial_psnr_db": round(plains[0]["psnr"][0], 4), "target_psnr_db": round(target, 4),
            "plain_fp32_seconds_30": round(t_plain, 5),
            "plain_fp32_psnr_at_30": [round(p["psnr"][30], 4) for p in plains],
            "plain_diverges": bool(target < plains[0]["psnr"][0]),
            "headline_path": head_path,
            "learned_seconds": None if t_lm is None else round(t_lm, 5),
            "speedup_vs_plain": None if not t_lm else round(t_plain / t_lm, 3),
            "runs": {k: per_path(rs) for k, rs in runs.items()},
            "psnr_curves": {k: [round(x, 3) for x in rs[0]["psnr"]] for k, rs in runs.items()},
        }
    head = starts["workload"]
    first = {name: first_sweep_ms(prec, use, use_damp=ud) for name, prec, use, ud in
             (("plain_fp32", 0, False, False), ("learned_fp32", 0, True, False), ("plain_mixed", 1, False, False),
              ("learned_mixed", 1, True, False), ("damping_mixed", 1, False, True),
              ("damping_scale_mixed", 1, True, True))}
    result = {
        "metric": "time to PSNR vs plain FP32 path (object workload)",
        "value": head["learned_seconds"], "unit": "s", "higher_is_better": False,
        "starts": starts,
        "first_sweep_ms": first,
        "network": {"objective": args.ttp_objective, "learned_trust": args.ttp_learned_trust,
                    "damping_objective": args.ttp_damping_objective + " (labels: the candidate rho minimising the "
                                         "all-view quadratic model; line: the same, each record weighted by the "
                                         "spread of that model over the candidates)",
                    "tiny_runs": args.ttp_runs, "shell_runs": args.ttp_shell, "shell_sweeps": args.ttp_shell_sweeps,
                    "records": tiny.n + shell.n,
                    "collect_s": round(t_collect, 2), "train_s": round(t_train, 2), "epochs": args.ttp_epochs,
                    "heldout": held_stats},
        "config": {"workload": "object: " + w["desc"], "primaries": "seeded permutation (seed 5)",
                   "psnr": "mean over all cameras of 10 log10(1 / MSE), images not clamped"},
        "dtype": "f32 (plain) / f32+f64 (mixed), network bf16 weights f32 accumulation",
        "data": "synthetic",
    }
    return result


# ----------------------------------------------------------------------------- oracle (CPU) arm

def oracle_group_pass_seconds(O, scene_h, cam, group, crop, ocfg, target_full):
    """Time one oracle group pass (render + loss derivatives + block assembly)
    on a crop x crop window in the image centre."""
    cw = synth.Camera(crop, crop, cam.fx, cam.fy, cam.cx - (cam.width // 2 - crop // 2),
                      cam.cy - (cam.height // 2 - crop // 2), cam.viewmat,
                      1.3 * 0.5 * cam.width / cam.fx, 1.3 * 0.5 * cam.height / cam.fy)
    y0, x0 = cam.height // 2 - crop // 2, cam.width // 2 - crop // 2
    tgt = target_full[:, y0:y0 + crop, x0:x0 + crop]
    t0 = time.perf_counter()
    img = O.render(scene_h, cw, ocfg)["image"]
    L = O.loss(img, tgt, ocfg)
    O.accum(group, scene_h, cw, cam, L["e"], L["h"], ocfg)
    return time.perf_counter() - t0


def subset_scene(scene, frac, seed=12):
    """Random subset of the Gaussians (the oracle's costs are linear in N)."""
    n = scene.n
    m = max(1, int(round(frac * n)))
    idx = np.sort(np.random.default_rng(seed).choice(n, m, replace=False))
    return synth.Scene(scene.mean[:, idx], scene.quat[:, idx], scene.scale[:, idx], scene.opacity[idx],
                       scene.sh[:, :, idx], scene.sh_degree)


def oracle_sweep_estimate(w, train_host, cams, group_list, small=1, big=12, frac=0.05):
    """Seconds per sweep of the oracle, extrapolated from timed samples: per
    group, a 1x1 crop (fixed cost: projecting every Gaussian as jets) and a
    big x big crop (adds the per-pixel cost), both on a random fraction `frac`
    of the Gaussians and scaled by 1/frac (brute-force compositing and the jet
    projection are linear in the Gaussian count); a sweep = sum over groups and
    the 4 views of fixed + per-pixel x pixels."""
    from oracle import oracle as O
    O.build()
    ocfg = O.default_config()
    scene_h = O.scene_handle(subset_scene(train_host, frac) if frac < 1 else train_host)
    cam = cams[0]
    tgt = synth.procedural_targets(1, cam.width, cam.height, seed=11)[0]
    P_full = cam.width * cam.height
    P_half = (cam.width // 2) * (cam.height // 2)
    per_group = {}
    t_start = time.perf_counter()
    for g in group_list:
        f = oracle_group_pass_seconds(O, scene_h, cam, g, small, ocfg, tgt)
        b = oracle_group_pass_seconds(O, scene_h, cam, g, big, ocfg, tgt)
        per_px = max(b - f, 0.0) / (big * big - small * small)
        per_group[g] = (f / frac, per_px / frac)
    spent = time.perf_counter() - t_start
    return per_group, spent, P_full, P_half


def sweep_seconds(per_group, P_full, P_half, K=3):
    tot = 0.0
    known = list(per_group.values())
    for g in range(5):
        f, px = per_group.get(g, (statistics.mean(x[0] for x in known), statistics.mean(x[1] for x in known)))
        tot += (f + px * P_full) + K * (f + px * P_half)
    return tot


def oracle_tiny_sweep_seconds():
    """One whole oracle sweep, timed, on the tiny workload (1,000 Gaussians, 4
    cameras 128x128, SH degree 0; primary 0, its 3 KNN secondaries, 5 groups):
    a measured figure beside the extrapolated one of the large workloads."""
    from oracle import oracle as O
    O.build()
    ocfg = O.default_config()
    w, gt, train, cams = make_workload("tiny")
    tg = np.stack([O.render(gt, c, ocfg)["image"] for c in cams])
    centres = np.stack([c.center() for c in cams])
    knn, _ = O.knn(centres, O.bounding_sphere(train), 3)
    t0 = time.perf_counter()
    O.sweep(train, cams, tg, knn, 0, ocfg)
    return time.perf_counter() - t0


def cpu_baseline(args, w, train_host, cams):
    per_group, spent, P_full, P_half = oracle_sweep_estimate(w, train_host, cams, range(5),
                                                             big=args.cpu_crop)
    t = sweep_seconds(per_group, P_full, P_half)
    tiny = oracle_tiny_sweep_seconds()
    return {"value": 1.0 / t, "unit": "sweeps/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"FP64 oracle (brute-force compositing, jet-derived blocks), every group on 1x1 and "
                       f"{args.cpu_crop}x{args.cpu_crop} centre crops of the primary view of the "
                       f"{args.workload} workload with a random 5% of its Gaussians; costs scaled by 20 "
                       f"(linear in N) and extrapolated to 1 full-res + 3 half-res views x 5 groups; "
                       f"{spent:.1f} s of CPU work"),
            "seconds_per_sweep": round(t, 1),
            "measured_tiny": {"workload": "tiny: " + WORKLOADS["tiny"]["desc"], "seconds_per_sweep": round(tiny, 3),
                              "sweeps_per_s": round(1.0 / tiny, 4),
                              "what": "one whole oracle sweep (5 groups x 1 primary + 3 secondaries), timed"}}


def run_reference(args):
    """The oracle as the reference arm.  A whole oracle sweep of this workload
    takes hours, so each step is a bounded sample: one group (cycling) on a
    1x1 and a ref_crop x ref_crop centre crop of the primary view with a random
    5% of the Gaussians.  ms_per_step is the measured time of those samples;
    value is the sweeps/s that the samples extrapolate to (costs scaled by 20,
    linear in N, and by the views' pixel counts), with the extrapolated seconds
    per sweep in its own field."""
    w, gt_host, train_host, cams = make_workload(args.workload)
    samples = {}
    from oracle import oracle as O  # noqa: F401
    step_s = []
    t0 = time.perf_counter()
    for i in range(args.warmup + args.steps):
        g = i % 5
        pg, spent, P_full, P_half = oracle_sweep_estimate(w, train_host, cams, [g], big=args.ref_crop)
        if i >= args.warmup:
            samples.setdefault(g, []).append(pg[g])
            step_s.append(spent)
    per_group = {g: (statistics.mean(x[0] for x in v), statistics.mean(x[1] for x in v)) for g, v in samples.items()}
    t = sweep_seconds(per_group, P_full, P_half)
    value = 1.0 / t
    sample = (f"each step: one group (cycling) on 1x1 and {args.ref_crop}x{args.ref_crop} centre crops of the "
              f"primary view with a random 5% of the Gaussians (measured: ms_per_step); value: those costs "
              f"scaled by 20 and extrapolated to a full sweep (extrapolated_seconds_per_sweep); "
              f"{time.perf_counter() - t0:.1f} s total")
    res = {"impl": "reference", "metric": "Newton sweeps/s (1 primary + 3 secondaries, 5 attribute groups)",
           "value": value, "unit": "sweeps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1e3 * statistics.mean(step_s), 1), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "extrapolated_seconds_per_sweep": round(t, 1),
           "config": {"workload": f"{args.workload}: {w['desc']}", "gaussians": w["n"], "cameras": len(cams),
                      "width": w["width"], "height": w["height"], "sh_degree": w["sh"]},
           "cpu_baseline": {"value": value, "unit": "sweeps/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return res


KERNEL_REV = "accum-v15"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gs2", choices=["gs2", "reference"])
    ap.add_argument("--workload", default="scene", choices=list(WORKLOADS) + ["batched"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-crop", type=int, default=12)
    ap.add_argument("--ref-crop", type=int, default=8)
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1],
                    help="1 (default): the precision form of the scene workload (FP64 accumulation of FP32 "
                         "partials, FP64 re-solve of blocks with condition estimate > 1e6); 0: FP32 only")
    ap.add_argument("--no-fp32-path", action="store_true", help="skip timing the FP32 path beside the mixed one")
    ap.add_argument("--no-det-path", action="store_true", help="skip timing the deterministic mode")
    ap.add_argument("--cams", type=int, default=0, help="use only the first N cameras (profiling captures)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default kernel tuning")
    ap.add_argument("--accum-px", type=int, default=0, choices=[0, 2, 4],
                    help="pixels per thread of the position accumulation (overrides the tuning; 0: keep)")
    ap.add_argument("--accum-split", type=int, default=-1,
                    help="list entries per work item of the split accumulation (overrides the tuning; 0: off, "
                         "-1: keep)")
    ap.add_argument("--batched-only", default="",
                    help="comma-separated indices of the batched workload's scenes to run (profiling captures)")
    ap.add_argument("--graph", type=int, default=1, choices=[0, 1],
                    help="1: time sweeps as a CUDA graph re-captured per sweep (one-scene gs2_batch); 0: eager")
    ap.add_argument("--variants", action="store_true",
                    help="method variants on the object workload: K in {0, 3, 8}, colour-first order, Gauss-Newton")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip timing the single-render (Jacobi over groups) variant beside the headline")
    ap.add_argument("--gd", action="store_true",
                    help="first-order baseline (gradient steps) on the object workload vs one Newton sweep")
    ap.add_argument("--variants-n", type=int, default=0, help="Gaussians of the object shell for --variants")
    ap.add_argument("--variants-sd", type=float, default=0.0,
                    help="perturbation of the start's means for --variants (default 0.02, the workload's)")
    ap.add_argument("--variants-only", default="", help="comma-separated variant names for --variants")
    ap.add_argument("--variants-cfg", default="", help="config overrides for every variant, key=value,...")
    ap.add_argument("--ttp", action="store_true", help="time to PSNR on the object workload (learned + mixed "
                                                       "vs plain FP32), one JSON line")
    ap.add_argument("--ttp-runs", type=int, default=1000, help="tiny-scene record runs")
    ap.add_argument("--ttp-shell", type=int, default=24, help="shell-scene record runs")
    ap.add_argument("--ttp-shell-sweeps", type=int, default=4, help="logged sweeps per shell-scene record run")
    ap.add_argument("--ttp-epochs", type=int, default=3)
    ap.add_argument("--ttp-max", type=int, default=60)
    ap.add_argument("--ttp-learned-trust", type=float, default=1.0,
                    help="learned_trust of the learned paths (the learned step may reach this many trust radii)")
    ap.add_argument("--ttp-reps", type=int, default=3,
                    help="runs of every path from each start (medians and spread are reported)")
    ap.add_argument("--ttp-paths", default="learned_mixed,damping_mixed,damping_scale_mixed,plain_mixed",
                    help="paths run against the plain FP32 path: learned_mixed, learned_fp32, learned_mixed_radii_x2, "
                         "damping_mixed, damping_scale_mixed, plain_mixed")
    ap.add_argument("--ttp-damping-objective", default="line", choices=["line", "labels"],
                    help="damping network: line = label loss weighted per record by the spread of the all-view "
                         "quadratic model over the candidates; labels = unweighted")
    ap.add_argument("--ttp-objective", default="line", choices=["line", "labels"],
                    help="training loss of the step-scale network")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "gs2" else args.warmup

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.ttp:
        if rank == 0:
            print(json.dumps(time_to_psnr(args)), flush=True)
        return
    if args.variants:
        if rank == 0:
            print(json.dumps(method_variants(args)), flush=True)
        return
    if args.gd:
        if rank == 0:
            print(json.dumps(gd_baseline(args)), flush=True)
        return
    if args.workload == "batched" and args.impl == "gs2":
        if rank == 0:
            print(json.dumps(run_batched(args)), flush=True)
        return

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    result, (w, train_host, cams) = run_gpu(args, rank, world, local_rank)
    if rank == 0:
        if not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline(args, w, train_host, cams)
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
