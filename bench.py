#!/usr/bin/env python
"""Benchmark: differentiable textured-2DGS training step (forward + L1 loss +
backward) on 200k textured splats at 800x800, reported as Mpix/s.

Workload (synthetic, seeded; stands in for the paper's Shiny Blender
object captures): 160k splats on a unit sphere + 40k in a [-1,1]^3 box,
8x8 texels x 8 channels, 100 cameras on a radius-4 Fibonacci sphere, 800x800,
L1 loss to seeded U[0,1] targets, 32x32 cube + 8x8 irradiance + 128x128 BRDF
table.  One step = four views (--views-per-step) in one launch sequence:
binning, render (with saved state), the four losses, backward.  Gradients
accumulate over the views and steps (a multi-view gradient accumulation), so
every view gets the full forward and backward; consecutive steps alternate
between two CUDA streams (--no-pipeline: one).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank renders its own views (replicas, no collective on
the data path); the time is the max over ranks.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpix/s fwd+bwd at 200k splats 800²; served-view p50/p99 latency vs plain"
UNIT = "Mpix/s"
N_SPLATS, T_TEX, RES, N_CAMS = 200_000, 8, 800, 100
VIEWS_PER_STEP = 4  # views rendered and differentiated per launch sequence (one step)
PREC_TILES = 16  # seeded covered 16x16 tiles (4096 px) per error view scored against the FP64 oracle
FP32_LANES_PER_SM = 128  # FP32 FMA lanes per SM on this architecture (sm_100 family)

# FP32 operations per fragment of the algorithm (FMA = 2): every evaluated
# (pixel, splat) pair costs the homography (6 FMA, a reciprocal, 2 mul) and the
# support cut; every blended fragment adds kernel/alpha (8), texel setup (8),
# the 8-channel bilinear filter (72 + weights), normal mapping (15) and
# blending (19); the backward recomputes that and adds the adjoint (~260: the
# tangent-normal pull-back, the corner dot products, alpha / (u, v) / depth
# derivatives, the frame torque and the per-fragment texel and record sums).
# Shading costs 150 per pixel forward (fused into the forward rasteriser) and
# 400 per pixel in the adjoint (its own kernel).
FLOP_EVAL = 15
FLOP_BLEND_FWD = 124
FLOP_BLEND_BWD = 124 + 260
FLOP_SHADE_FWD = 150
FLOP_SHADE_BWD = 400


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-tiles", type=int, default=6, help="tiles of the oracle CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--views-per-step", type=int, default=VIEWS_PER_STEP,
                    help="views batched into one launch sequence per step")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="one stream: each view's forward waits for the previous view's backward")
    ap.add_argument("--no-serve", action="store_true", help="skip the served-view latency measurement")
    ap.add_argument("--serve-only", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-warmup", type=int, default=200)
    ap.add_argument("--serve-rate", type=float, default=1.0, help="arrival rate / plain saturated fps")
    ap.add_argument("--serve-sweep", type=float, nargs="*", default=[0.5, 0.8, 1.0, 1.5],
                    help="further arrival-rate factors timed after the headline one")
    ap.add_argument("--no-large", action="store_true", help="skip the 3M-splat training-step measurement")
    ap.add_argument("--large-only", action="store_true")
    ap.add_argument("--large-steps", type=int, default=10)
    ap.add_argument("--large-warmup", type=int, default=3)
    ap.add_argument("--no-precision", action="store_true", help="skip the reduced-precision atlas measurement")
    ap.add_argument("--precision-only", action="store_true")
    ap.add_argument("--no-sampling", action="store_true", help="skip the texture-sampler comparison (Table 3 shape)")
    ap.add_argument("--sampling-only", action="store_true")
    ap.add_argument("--sampling-views", type=int, default=40)
    ap.add_argument("--no-image-loss", action="store_true", help="skip the L1 + D-SSIM timing after the step")
    ap.add_argument("--no-fp32-probe", action="store_true", help="skip the FP32 rate probe after the step")
    ap.add_argument("--packing-probe", action="store_true",
                    help="one hardware-atlas render per chart packing (splat id, Morton), for profiling")
    ap.add_argument("--hbm-kernels-only", action="store_true",
                    help="time the atlas pack and Adam alone on 1 GiB of float32 (for profiling)")
    ap.add_argument("--no-features", action="store_true",
                    help="skip the indirect-light / two-component-normal step timings")
    ap.add_argument("--features-only", action="store_true")
    ap.add_argument("--feature-steps", type=int, default=20)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_views(rank: int, n_needed: int) -> list:
    """Camera (and target) indices rank `rank` renders: each rank starts at
    its own offset of the camera set, so replicas work on different views."""
    return [(rank * 7 + i) % N_CAMS for i in range(n_needed)]


def max_over_ranks(ms: float, pg, device) -> float:
    """The slowest rank's time: the whole job's time for `value`."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if pg is not None:
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(world: int, steps: int, ms_max: float, views: int = 1) -> float:
    """Whole-job Mpix/s: every rank renders `steps` steps of `views` views of RES x RES."""
    return world * steps * views * RES * RES / 1e6 / (ms_max / 1e3)


def workload_config(world: int, pipelined: bool = True, views: int = VIEWS_PER_STEP) -> dict:
    return {"workload": "cfg1: 200k textured splats (160k sphere + 40k box), 8x8 texels x 8 ch, "
                        "800x800, forward + L1 loss + backward per view",
            "splats": N_SPLATS, "texels": f"{T_TEX}x{T_TEX}x8 f32", "resolution": f"{RES}x{RES}",
            "views_per_step": views,
            "batching": (f"{views} views (cameras i..i+{views - 1} of the 100) per launch sequence: one binning, "
                         "forward, loss and backward pass over all their tiles" if views > 1 else "one view per step"),
            "parallelism": f"replicas x{world}",
            "streams": ("2: step i+1's binning and forward overlap step i's backward" if pipelined
                        else "1: steps in sequence"),
            "l2": "inputs larger than L2 (texel atlas 410 MB, records+pairs ~90 MB per view)"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 20 ms around the
    timed region; samples carry nvidia-smi's timestamp, and the summary is
    taken over those inside the timed window [t0, t1] (host wall clock,
    both ends after a device synchronisation)."""

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        # the timed region starts only once the sampler is producing
        deadline = time.time() + 5.0
        while self.proc is not None and time.time() < deadline:
            if os.path.exists(self.path) and os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self, t0: float, t1: float) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.05)  # one more sample past the end of the window
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        return summarise_clocks(lines, t0, t1)


def summarise_clocks(lines, t0: float, t1: float, interval_ms: int = 20) -> dict:
    """Median SM clock, maximum clock and active slowdown reasons of the
    nvidia-smi samples (timestamp first) inside [t0, t1] (all samples if
    none fell inside)."""
    import datetime
    rows = []
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 10:
            continue
        try:
            ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            rows.append((ts, float(parts[2]), float(parts[3]),
                         {nm for nm, val in zip(names, parts[6:10]) if val.lower() == "active"}))
        except ValueError:
            continue
    inside = [r for r in rows if t0 <= r[0] <= t1]
    use = inside if inside else rows
    reasons = set().union(*[r[3] for r in use]) if use else set()
    return {"sm_mhz": statistics.median([r[1] for r in use]) if use else None,
            "sm_max_mhz": max(r[2] for r in use) if use else None,
            "reasons": sorted(reasons), "samples": len(inside), "samples_total": len(rows),
            "window_s": round(t1 - t0, 4), "interval_ms": interval_ms}


def build_workload(seed_cams=0):
    import scenegen as sg
    scene = sg.make_scene(1)
    env = sg.make_env(1, cube_res=32, levels=1, irr_res=8, lut_res=128)
    cams = sg.fibonacci_cameras(N_CAMS, 4.0, RES, RES)
    return scene, env, cams


# ----------------------------------------------------------------------------
def cpu_oracle_sample(scene, env, cam, n_tiles: int, seed: int = 0):
    """Times the FP64 oracle (forward + autograd backward) on the n_tiles
    seeded random non-empty tiles of one view.  Returns (Mpix/s, seconds, threads, pixels)."""
    import numpy as np
    import torch

    import scenegen as sg
    from oracle import grad as G
    from oracle import keys as K

    kl = K.build_keys(scene, cam)
    lens = kl["tile_ranges"][:, 1] - kl["tile_ranges"][:, 0]
    rng = np.random.default_rng(seed)
    busy = np.nonzero(lens > 0)[0]
    tiles = sorted(rng.choice(busy, size=min(n_tiles, busy.size), replace=False).tolist())
    tgt = sg.make_target(seed, RES, RES)
    dL = np.sign(rng.normal(size=tgt.shape)) / (3.0 * RES * RES)
    t0 = time.perf_counter()
    G.render_grads(scene, cam, env, dL, tiles=tiles, keylist=kl)
    dt = time.perf_counter() - t0
    px = 256 * len(tiles)
    return px / dt / 1e6, dt, torch.get_num_threads(), px, (tiles, kl)


def parity_sample(scene, env, cam, tiles, kl, gpu_rgba):
    """The GPU image of the timed workload against the oracle on the sampled
    tiles (untimed): max-abs error over pixels with an admissible oracle
    result (the definition's, or with the one threshold decision that lies
    within FP32 error of flipping flipped), and the masked fraction (pixels
    with several such decisions)."""
    import numpy as np

    from oracle import render as R
    ref = R.render(scene, cam, env, tiles=tiles, keylist=kl)
    g = gpu_rgba.detach().cpu().numpy().astype(np.float64)
    tiles_x = kl["view"]["tiles_x"]
    sel = np.zeros(g.shape[:2], dtype=bool)
    for t in tiles:
        ty, tx = divmod(int(t), tiles_x)
        sel[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16] = True
    r, ra = ref["rgba"].detach().numpy(), ref["alt"]["rgba"].numpy()
    amb, alt = ref["ambiguous"].numpy(), ref["alt"]["mask"].numpy()
    err = np.minimum(np.abs(g - r).max(-1), np.abs(g - ra).max(-1))
    ok = sel & ~amb
    return {"pixels": int(sel.sum()), "max_abs_err": float(err[ok].max()) if ok.any() else 0.0,
            "tolerance": 1e-4, "masked": int((amb & sel).sum()), "masked_frac": float((amb & sel).sum() / sel.sum()),
            "two_results": int((alt & sel).sum()),
            "note": "GPU image of the first timed view vs the FP64 oracle on the CPU-baseline tiles"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import torch
    scene, env, cams = build_workload()
    vals, secs = [], []
    for i in range(args.warmup + args.steps):
        v, dt, thr, px, _ = cpu_oracle_sample(scene, env, cams[i % N_CAMS], max(1, args.cpu_tiles // 3), seed=i)
        if i >= args.warmup:
            vals.append(v)
            secs.append(dt)
    total_px = 256 * max(1, args.cpu_tiles // 3) * args.steps
    value = total_px / sum(secs) / 1e6
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": dict(workload_config(world),
                           sample=f"{max(1, args.cpu_tiles // 3)} random non-empty 16x16 tiles per step"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": f"{max(1, args.cpu_tiles // 3)} random non-empty tiles of each view, fwd+autograd bwd, FP64"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    import paper_2506_13348_b300 as P
    from paper_2506_13348_b300 import _lib
    import scenegen as sg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    scene, env, cams = build_workload()
    sc = P.Scene.from_arrays(scene, env, device=local)
    B = max(1, args.views_per_step)
    n_needed = min(N_CAMS, (args.warmup + args.steps) * B)
    views = rank_views(rank, n_needed)
    my_cams = [cams[i] for i in views]
    targets = [torch.from_numpy(sg.make_target(i, RES, RES)).to(dev) for i in views]
    out = torch.empty(RES, RES, 4, dtype=torch.float32, device=dev)
    grads = P.zero_grads(sc)
    stream = torch.cuda.current_stream()
    # a step renders B views in one launch sequence (their tiles form one
    # grid per kernel); steps alternate between two streams: step i+1's
    # binning and forward overlap step i's backward (gradients accumulate
    # with atomics, so the two backwards may also overlap); each stream has
    # its own images, losses and gradient images
    streams = [stream] + ([torch.cuda.Stream(device=dev)] if not args.no_pipeline else [])
    bufs = [([torch.empty_like(out) for _ in range(B)], [torch.empty_like(out) for _ in range(B)],
             torch.zeros(B, dtype=torch.float32, device=dev)) for _ in streams]

    def step(i, serial=False):
        k = 0 if serial else i % len(streams)
        st, (o, d, l) = streams[k], bufs[k]
        vi = [(i * B + j) % n_needed for j in range(B)]
        if B == 1:
            _, saved = P.render(sc, my_cams[vi[0]], out=o[0], save=True, stream=st)
        else:
            _, saved = P.render_views([sc] * B, [my_cams[v] for v in vi], outs=o, save=True, stream=st)
        for j, v in enumerate(vi):
            P.l1_loss(o[j], targets[v], l[j:j + 1], d[j], stream=st)
        P.render_backward(saved, d, grads, stream=st)
        saved.release()

    def timed(steps, serial):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for s2 in streams[1:]:
            s2.wait_event(e0)
        for i in range(steps):
            step(args.warmup + i, serial)
        for s2 in streams[1:]:
            stream.wait_stream(s2)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    t_w0 = time.time()
    l0 = _lib.launch_count()
    ms = timed(args.steps, serial=False)
    launches = _lib.launch_count() - l0
    t_w1 = time.time()  # timed() ends with a device synchronisation
    if pg:
        pg.barrier()
    # the same steps once more on one stream with per-stage CUDA events: the
    # kernels' own durations (the roofline) without the other view's work
    # sharing the SMs
    _lib.profile_enable(True)
    _lib.profile_report()
    ms_serial = timed(args.steps, serial=True)
    stages = _lib.profile_report()
    _lib.profile_enable(False)
    clocks = sampler.stop(t_w0, t_w1)
    ms_max = max_over_ranks(ms, pg, dev)
    value = aggregate_value(world, args.steps, ms_max, B)

    # fragment statistics of a few of the timed views (untimed pass)
    fr = {"n_pairs": 0, "n_evaluated": 0, "n_blended": 0, "n_visible": 0, "n_texels_read": 0, "n_items_blended": 0}
    nstat = 4
    for i in range(nstat):
        _, saved = P.render(sc, my_cams[(args.warmup + i) % n_needed], out=out, save=True)
        s = saved.frag_stats()
        saved.release()
        for k in fr:
            fr[k] += s[k] / nstat
    npix = RES * RES
    # per launch: each rasteriser launch covers the step's B views
    flops_fwd = B * (FLOP_EVAL * fr["n_evaluated"] + FLOP_BLEND_FWD * fr["n_blended"] + FLOP_SHADE_FWD * npix)
    # the shading adjoint (FLOP_SHADE_BWD per pixel) runs in k_shade_bwd, not in the rasteriser
    flops_bwd = B * (FLOP_EVAL * fr["n_evaluated"] + FLOP_BLEND_BWD * fr["n_blended"])
    peaks, peak_kind = load_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = n_sm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s
    stage_ms = {k: v[1] / max(1, v[0]) for k, v in stages.items()}
    dom = max(("raster_fwd", "raster_bwd"), key=lambda k: stages.get(k, (0, 0.0))[1])
    dom_ms = stage_ms.get(dom, float("nan"))
    dom_flops = flops_bwd if dom == "raster_bwd" else flops_fwd
    achieved = dom_flops / (dom_ms / 1e3) / 1e12
    traffic = read_traffic(dom, B)
    rbytes = {k: B * v for k, v in raster_bytes(fr, npix).items()}
    # measured FP32 FMA rate of this GPU (after the timed region): context for
    # the derived peak above
    meas_scalar, meas_paired = (float("nan"), float("nan")) if args.no_fp32_probe else _lib.measure_fp32_peak(local)

    # HBM-side stages against the measured copy rate (algorithmic bytes / time)
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
    # per launch: every stage covers the step's B views except the loss (one launch per view)
    sb = {k: (v if k == "l1_loss" else B * v)
          for k, v in stage_bytes(len(scene["opacity"]), fr["n_pairs"], npix, ((RES + 15) // 16) ** 2).items()}
    stage_fracs = {k: round(b / (stage_ms[k] / 1e3) / 1e9 / hbm_peak, 3) for k, b in sb.items() if k in stage_ms}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(world, not args.no_pipeline, B),
            "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": fp32_peak,
                         "timing": "kernel's own CUDA events in a second timed pass of the same steps on one stream",
                         "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": traffic,
                         "peak_note": f"FP32 FMA peak {n_sm} SMs (device) x {FP32_LANES_PER_SM} lanes x 2 x {sm_mhz:.0f} MHz "
                                      f"(clock from {peak_kind} peaks)",
                         "flops_per_launch": dom_flops, "ms_per_launch": dom_ms,
                         "alg_bytes_per_launch": rbytes[dom],
                         "traffic_over_alg_bytes": traffic / rbytes[dom] if traffic else None,
                         "peak_measured": None if args.no_fp32_probe else {
                             "scalar_fma_tflops": round(meas_scalar, 2), "paired_fma_tflops": round(meas_paired, 2),
                             "frac_of_measured_scalar": achieved / meas_scalar}},
            "roofline_fwd": roofline_other(dom, stage_ms, flops_fwd, flops_bwd, fp32_peak, meas_scalar, rbytes, B),
            "serial_ms_per_step": ms_serial / args.steps,
            "stages_ms": {k: round(v, 4) for k, v in stage_ms.items()},
            "stage_hbm_frac": stage_fracs,
            "fragments_per_view": {k: int(v) for k, v in fr.items()},
            "gpu_launches": int(launches),
            "clocks": clocks}
    if not args.no_image_loss:
        line["image_loss"] = time_image_loss(P, out, targets[0], dev)
    if not args.no_e2e:
        line["e2e"] = run_e2e(P, sc, my_cams, n_needed, args, dev, pg, world)
    par_img = None
    if rank == 0 and not args.no_cpu_baseline:  # the image the parity sample checks (untimed)
        par_img = P.render(sc, my_cams[0])[0].cpu()
    if rank == 0 and not args.no_serve:
        del grads
        sc.close()
        torch.cuda.empty_cache()
        line["serving"] = run_serving(args, local)
    if rank == 0 and not args.no_large:
        line["large_scene"] = run_large_scene(args, local)
    prec_inputs = None
    if rank == 0 and not args.no_precision:
        line["precision"] = run_precision(args, local)
        prec_inputs = line["precision"].pop("_oracle_inputs")
    if rank == 0 and not args.no_sampling:
        line["texture_sampling"] = run_sampling(args, local)
    if rank == 0 and not args.no_features:
        line["features"] = run_features(args, local)
    if rank == 0 and not args.no_cpu_baseline:
        v, dt, thr, px, (tiles, kl) = cpu_oracle_sample(scene, env, my_cams[0], args.cpu_tiles)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
                                "sample": f"{args.cpu_tiles} random non-empty 16x16 tiles ({px} px) of one 800x800 view, "
                                          f"FP64 forward + autograd backward, {dt:.1f} s"}
        line["parity_sample"] = parity_sample(scene, env, my_cams[0], tiles, kl, par_img)
        if prec_inputs is not None:
            line["precision"]["vs_fp64_oracle"] = precision_vs_oracle(prec_inputs)
    if rank == 0:
        print(json.dumps(line))
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def roofline_other(dom, stage_ms, flops_fwd, flops_bwd, fp32_peak, meas_scalar, rbytes, views):
    """The roofline of the rasteriser that is not the dominant kernel (the
    forward, normally), on the same FLOP model, peak and per-stage event
    timing as the dominant one."""
    other = "raster_fwd" if dom == "raster_bwd" else "raster_bwd"
    ms = stage_ms.get(other, float("nan"))
    flops = flops_fwd if other == "raster_fwd" else flops_bwd
    achieved = flops / (ms / 1e3) / 1e12
    traffic = read_traffic(other, views)
    return {"bound": "alu", "kernel": other, "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": traffic, "flops_per_launch": flops,
            "ms_per_launch": ms, "alg_bytes_per_launch": rbytes[other],
            "traffic_over_alg_bytes": traffic / rbytes[other] if traffic else None,
            "frac_of_measured_scalar": achieved / meas_scalar if meas_scalar == meas_scalar else None}


def run_serving(args, device):
    """Served-view latency: 3 resident scenes (200k / 500k / 1M splats, 8x8
    texels), Poisson arrivals of views at random cameras (radius U[3.5, 5])
    and resolutions drawn from {400x400, 800x800, 1280x720, 1920x1080}.
    'plain' = FP32 atlas, one request at a time, FIFO on one stream;
    'served' = BF16 atlas, continuous batching (2 streams, up to 8 views per
    batch).  Both see the same arrival schedule at rate = rate_factor x the
    plain renderer's saturated throughput; the headline factor (1.0) is
    reported in full and the sweep (0.5, 0.8, 1.0, 1.5) as p50 / p99 / fps.
    200 warm-up requests, then 2000 measured ones per run."""
    import threading

    import numpy as np
    import torch

    import paper_2506_13348_b300 as P
    import scenegen as sg

    env = sg.make_env(3, cube_res=32, levels=1, irr_res=8, lut_res=128)
    sizes = [200_000, 500_000, 1_000_000]
    plain_sc, served_sc = [], []
    for i, n in enumerate(sizes):
        s = sg.make_scene(1, n=n, T=8, seed=300 + i)
        plain_sc.append(P.Scene.from_arrays(s, env, device=device, store="f32"))
        served_sc.append(P.Scene.from_arrays(s, env, device=device, store="bf16"))
        del s
    rng = np.random.default_rng(3)
    nreq = args.serve_requests + args.serve_warmup
    res = [(400, 400), (800, 800), (1280, 720), (1920, 1080)]
    cams = sg.random_sphere_cameras(rng, nreq, 3.5, 5.0, res)
    which = rng.integers(0, 3, size=nreq)

    def run(server, scenes, gaps):
        # warm-up requests first (all collected), then the statistics are
        # reset and the measured requests follow on the same schedule
        def phase(lo, hi):
            tickets = [None] * nreq

            def consumer():
                for i in range(lo, hi):
                    while tickets[i] is None:
                        time.sleep(0.0002)
                    server.wait(tickets[i], None, timeout_s=120.0)

            th = threading.Thread(target=consumer)
            th.start()
            t_next = time.perf_counter()
            for i in range(lo, hi):
                if gaps is not None:
                    t_next += gaps[i]
                    while True:
                        d = t_next - time.perf_counter()
                        if d <= 0:
                            break
                        time.sleep(min(d, 0.001) if d > 0.0015 else 0)
                tickets[i] = server.submit(scenes[which[i]], cams[i])
            th.join()

        phase(0, args.serve_warmup)
        server.reset_stats()
        phase(args.serve_warmup, nreq)
        return server.stats()

    arena = 24 << 30
    keep = ("p50_ms", "p99_ms", "mean_ms", "fps", "mpix_per_s", "mean_batch", "completed", "rejected")
    plain = P.Server(device=device, arena_bytes=arena, n_streams=1, max_batch=1)
    served = P.Server(device=device, arena_bytes=arena, n_streams=2, max_batch=8)
    sat = run(plain, plain_sc, None)  # all at once: saturated FIFO throughput
    s_sat = run(served, served_sc, None)
    # the headline rate, then the other arrival rates of the sweep (the same
    # Poisson schedule scaled), each for both servers
    factors = [args.serve_rate] + [f for f in args.serve_sweep if f != args.serve_rate]
    sweep = {}
    for f in factors:
        rate = f * sat["fps"]
        gaps = np.random.default_rng(33).exponential(1.0 / rate, size=nreq)
        p = run(plain, plain_sc, gaps)
        s = run(served, served_sc, gaps)
        sweep[f"{f:g}"] = {"arrival_rate_fps": rate, "plain_fp32_one_at_a_time": {k: p[k] for k in keep},
                           "served_bf16_batched": {k: s[k] for k in keep}}
    plain.close()
    served.close()
    for sc in plain_sc + served_sc:
        sc.close()
    head = sweep[f"{args.serve_rate:g}"]
    p, s, rate = head["plain_fp32_one_at_a_time"], head["served_bf16_batched"], head["arrival_rate_fps"]
    return {"workload": "cfg3: scenes of 200k/500k/1M splats (8x8 texels), Poisson arrivals, "
                        "resolutions {400^2, 800^2, 1280x720, 1920x1080}, radius U[3.5,5]",
            "requests": args.serve_requests, "warmup_requests": args.serve_warmup,
            "arrival_rate_fps": rate, "rate_factor": args.serve_rate,
            "plain_saturated_fps": sat["fps"], "served_saturated_fps": s_sat["fps"],
            "served_saturated_mean_batch": s_sat["mean_batch"],
            "plain_fp32_one_at_a_time": p, "served_bf16_batched": s,
            "rate_sweep": {f: {"plain_p50_ms": v["plain_fp32_one_at_a_time"]["p50_ms"],
                               "plain_p99_ms": v["plain_fp32_one_at_a_time"]["p99_ms"],
                               "served_p50_ms": v["served_bf16_batched"]["p50_ms"],
                               "served_p99_ms": v["served_bf16_batched"]["p99_ms"],
                               "plain_fps": v["plain_fp32_one_at_a_time"]["fps"],
                               "served_fps": v["served_bf16_batched"]["fps"]} for f, v in sweep.items()}}


def run_precision(args, device):
    """Reduced-precision atlas: 500k sphere splats, 16x16 texels x 8
    channels, 1920x1080, 6-level 128 FP16 cube.  Per stored dtype (f32,
    bf16, f16): forward Mpix/s over 10 views, the atlas pack's bandwidth,
    and the storage error of the bf16 / f16 images against the f32 atlas's
    images of the same views (whole images of views 0 and 5; the f32 path is
    the one the parity tests hold within 1e-4 of the FP64 oracle)."""
    import numpy as np
    import torch

    import paper_2506_13348_b300 as P
    from paper_2506_13348_b300 import _lib
    import scenegen as sg

    dev = torch.device("cuda", device)
    geo = sg.make_scene(2, with_texels=False)
    tex = sg.scenes.texels_torch(len(geo["opacity"]), 16, seed=2, device=dev)  # the pack reads HBM
    env = sg.make_env(2, cube_res=128, levels=6, irr_res=16, lut_res=128)
    W, H = 1920, 1080
    cams = sg.fibonacci_cameras(10, 4.0, W, H)
    err_views = (0, 5)
    out = {"workload": "cfg2: 500k splats, 16x16 texels x 8 ch, 1920x1080, 6-level 128 FP16 cube, 10 views",
           "error_reference": "images of views 0 and 5 (RGB, every pixel) rendered from the f32 atlas"}
    # seeded samples of the error views -- PREC_TILES whole 16x16 tiles among
    # those the image covers -- scored against the FP64 oracle (fed the
    # float32 texels) in the CPU-baseline leg
    srng = np.random.default_rng(7)
    samp = {}
    got = {}
    img = torch.empty(H, W, 4, device=dev)
    peaks, peak_kind = load_peaks()
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    ref_imgs = {}
    for store in ("f32", "bf16", "f16"):
        sc = P.Scene(device)
        sc.upload_gaussians(geo["means"], geo["quats"], geo["scales"], geo["opacity"])
        _lib.profile_enable(True)
        _lib.profile_report()
        sc.upload_atlas(tex, store)
        st = _lib.profile_report()
        _lib.profile_enable(False)
        sc.upload_envmap(env, "f16")
        errs = []
        for ci in err_views:
            P.render(sc, cams[ci], out=img)
            if ci not in samp:
                tx_n, ty_n = (W + 15) // 16, (H + 15) // 16
                a = torch.nn.functional.pad(img[..., 3], (0, tx_n * 16 - W, 0, ty_n * 16 - H))
                cov = (a.reshape(ty_n, 16, tx_n, 16).amax(dim=(1, 3)) > 0).flatten().cpu().numpy()
                tiles = np.sort(srng.choice(np.nonzero(cov)[0], size=PREC_TILES, replace=False))
                ys, xs = np.divmod(tiles, tx_n)
                gy, gx = np.meshgrid(np.arange(16), np.arange(16), indexing="ij")
                px_ = (xs[:, None] * 16 + gx.ravel()[None]).ravel()
                py_ = (ys[:, None] * 16 + gy.ravel()[None]).ravel()
                keep = (px_ < W) & (py_ < H)
                samp[ci] = (tiles, px_[keep], py_[keep])
            _, px_, py_ = samp[ci]
            got[(store, ci)] = img[torch.from_numpy(py_).to(dev), torch.from_numpy(px_).to(dev)].cpu().numpy()
            if store == "f32":
                ref_imgs[ci] = img[..., :3].clone()
            else:
                errs.append((img[..., :3] - ref_imgs[ci]).abs().double().flatten())
        for i in range(2):
            P.render(sc, cams[i], out=img)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(len(cams)):
            P.render(sc, cams[i], out=img)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / len(cams)
        res = {"fwd_ms_per_view": ms, "fwd_mpix_per_s": W * H / 1e6 / (ms / 1e3)}
        if "atlas_pack" in st:  # bf16 / f16: 4 B read + 2 B written per channel
            pms = st["atlas_pack"][1] / max(1, st["atlas_pack"][0])
            gbs = tex.numel() * 6 / (pms / 1e3) / 1e9
            res.update(pack_ms=pms, pack_gb_per_s=gbs, pack_frac_of_hbm=gbs / hbm,
                       pack_peak=f"{hbm:.0f} GB/s ({peak_kind})")
        if errs:
            e = torch.cat(errs)
            mse = float((e * e).mean())
            res.update(max_abs_err=float(e.max()), mean_abs_err=float(e.mean()),
                       psnr_db=float(10 * np.log10(1.0 / mse)) if mse > 0 else None)
        out[store] = res
        sc.close()
    out["_oracle_inputs"] = dict(geo=geo, tex=tex.cpu().numpy(), env=env, cams=[cams[ci] for ci in err_views],
                                 views=list(err_views), samples=samp, got=got)
    del tex, ref_imgs
    torch.cuda.empty_cache()
    return out


def precision_vs_oracle(inp):
    """Each reduced-precision image's error against the FP64 oracle fed the
    float32 texels (the storage error), on PREC_TILES seeded whole tiles of
    each error view: max-abs, mean-abs and PSNR over RGB.  The f32 row is
    the renderer's own error against the oracle.  Pixels with several
    threshold decisions within FP32 error are left out (counted); where one
    decision is, the nearer admissible oracle result is used."""
    import numpy as np

    from oracle import keys as K
    from oracle import render as R
    geo, tex, env = inp["geo"], inp["tex"], inp["env"]
    env16 = dict(env, spec=[m.astype(np.float16).astype(np.float32) for m in env["spec"]],
                 irr=env["irr"].astype(np.float16).astype(np.float32))
    scene = dict(geo, texels=tex, T=tex.shape[1])
    res = {"tiles_per_view": PREC_TILES, "reference": "FP64 oracle, float32 texels, the FP16 cube the renderer reads; "
                                                       "RGB of every pixel of seeded covered 16x16 tiles"}
    t0 = time.perf_counter()
    params, envp = R.to_params(scene), R.env_params(env16)
    for ci, cam in zip(inp["views"], inp["cams"]):
        kl = K.build_keys(scene, cam)
        tiles, px, py = inp["samples"][ci]
        ref = R.render(scene, cam, env16, params=params, envp=envp, tiles=tiles, keylist=kl)
        r, a = ref["rgba"].detach().numpy()[py, px], ref["alt"]["rgba"].numpy()[py, px]
        amb = ref["ambiguous"].numpy()[py, px]
        row = {"pixels": int(px.size), "masked": int(amb.sum())}
        for store in ("f32", "bf16", "f16"):
            g = inp["got"][(store, ci)].astype(np.float64)
            e0, e1 = (g - r)[..., :3], (g - a)[..., :3]
            pick = (np.abs(e0).max(-1) <= np.abs(e1).max(-1))[:, None]
            e = np.where(pick, e0, e1)[~amb]
            mse = float((e * e).mean())
            row[store] = {"max_abs_err": float(np.abs(e).max()), "mean_abs_err": float(np.abs(e).mean()),
                          "psnr_db": float(10 * np.log10(1.0 / mse)) if mse > 0 else None}
        res[f"view{ci}"] = row
    res["oracle_seconds"] = time.perf_counter() - t0
    return res


def run_large_scene(args, device):
    """Large-scene training step: 3M splats in a 10^3 box (60% on 32
    spheres, 40% uniform), 8x8 texels stored in BF16 with float32 masters,
    4 views of 1600x1064 per step from a radius-12 Fibonacci set: batched
    forward, L1 loss, backward, Adam on geometry and texels (master ->
    stored atlas), in-place geometry update."""
    import torch

    import paper_2506_13348_b300 as P
    import scenegen as sg

    dev = torch.device("cuda", device)
    torch.cuda.reset_peak_memory_stats(dev)
    geo = sg.make_scene(4, with_texels=False)
    n = len(geo["opacity"])
    tex = sg.scenes.texels_torch(n, 8, seed=4, device=dev)
    env = sg.make_env(4, cube_res=32, levels=1, irr_res=8, lut_res=128)
    sc = P.Scene.from_arrays(dict(geo, texels=tex), env, device=device, store="bf16")
    tr = P.Trainer(sc, dict(geo, texels=tex), store="bf16")
    del tex
    W, H, V = 1600, 1064, 4
    cams = sg.fibonacci_cameras(40, 12.0, W, H)
    targets = [torch.from_numpy(sg.make_target(i, W, H)).to(dev) for i in range(V)]
    outs = [torch.empty(H, W, 4, device=dev) for _ in range(V)]
    dls = [torch.empty_like(o) for o in outs]
    for i in range(args.large_warmup):
        tr.step(cams[(i * V) % 40:(i * V) % 40 + V], targets, outs, dls)
    torch.cuda.synchronize()
    from paper_2506_13348_b300 import _lib
    _lib.profile_enable(True)
    _lib.profile_report()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(args.large_steps):
        j = ((args.large_warmup + i) * V) % 40
        tr.step(cams[j:j + V], targets, outs, dls)
    e1.record()
    torch.cuda.synchronize()
    st = _lib.profile_report()
    _lib.profile_enable(False)
    ms = e0.elapsed_time(e1) / args.large_steps
    # per step: stage totals; Adam moves, per parameter, p g m v in (16 B), p m v
    # out and g zeroed (16 B), plus the 2-byte stored copy of each texel
    stage_ms = {k: round(v[1] / args.large_steps, 3) for k, v in st.items()}
    n_tex = n * 8 * 8 * 8
    n_geo = n * (3 + 4 + 2 + 1)
    adam_bytes = (n_tex + n_geo) * 32 + n_tex * 2
    peaks, peak_kind = load_peaks()
    adam_ms = stage_ms.get("adam", float("nan"))
    adam_gbs = adam_bytes / (adam_ms / 1e3) / 1e9
    peak = torch.cuda.max_memory_allocated(dev) / 1e9
    free, total = torch.cuda.mem_get_info(dev)
    out = {"workload": "cfg4: 3M splats in [-5,5]^3 (60% on 32 spheres, 40% uniform), 8x8 texels BF16 with "
                       "FP32 masters + Adam, 4 views of 1600x1064 per step",
           "splats": n, "steps": args.large_steps, "ms_per_step": ms,
           "mpix_per_s": V * W * H / 1e6 / (ms / 1e3),
           "torch_peak_alloc_gb": peak, "device_used_gb": (total - free) / 1e9,
           "stages_ms_per_step": stage_ms,
           "adam": {"ms_per_step": adam_ms, "bytes_per_step": adam_bytes, "gb_per_s": adam_gbs,
                    "frac_of_hbm": adam_gbs / float(peaks.get("hbm_gbs", 6400.0)), "peak": peak_kind}}
    # the HBM-side stages of a step against their algorithmic bytes (the
    # pair count of one untimed batch of the step's views)
    _, saved = P.render_views([sc] * V, cams[:V], outs=outs, save=True)
    K = saved.sizes()[0]
    saved.release()
    tiles = V * ((W + 15) // 16) * ((H + 15) // 16)
    sb = stage_bytes(V * n, K, V * W * H, tiles)
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    out["pairs_per_step"] = K
    out["stage_hbm_frac"] = {k: round(b / (stage_ms[k] / 1e3) / 1e9 / hbm, 3) for k, b in sb.items()
                             if stage_ms.get(k, 0) > 0}
    sc.close()
    del tr
    torch.cuda.empty_cache()
    return out


def time_image_loss(P, img, target, dev, reps=50):
    """The paper's image loss (0.8 L1 + 0.2 D-SSIM, Sec. 3.6) with its
    gradient on one 800x800 image, beside the L1 loss the timed step uses.
    Algorithmic traffic 152 B per pixel: the two images read twice (64 B),
    nine derivative maps written and read (72 B), the gradient written (16 B)."""
    import torch
    loss = torch.zeros(1, device=dev)
    grad = torch.empty_like(img)

    def t(fn):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms = t(lambda: P.image_loss(img, target, loss, grad, 0.2))
    ms_l1 = t(lambda: P.l1_loss(img, target, loss, grad))
    npx = img.shape[0] * img.shape[1]
    return {"l1_dssim_ms": ms, "l1_ms": ms_l1, "l1_dssim_gb_per_s": 152.0 * npx / (ms / 1e3) / 1e9}


def run_e2e(P, sc, cams, n_needed, args, dev, pg, world):
    """Same step through the public API with host buffers: each step's B
    target images go host->device from pinned memory and their B losses come
    back.  The copies run on a side stream into one of two sets of device
    buffers and overlap the render; the loss kernels wait for them.  Every
    copy is issued after the start event and consumed before the end event,
    so all of them are inside the timed region."""
    import torch

    import scenegen as sg
    B = max(1, args.views_per_step)
    host_t = [torch.from_numpy(sg.make_target(i, RES, RES)).pin_memory() for i in range(min(8, n_needed))]
    stream = torch.cuda.current_stream()
    # as the timed loop: steps alternate between the compute streams; per
    # stream B device targets, images and gradient images, B losses and
    # their pinned host copy
    streams = [stream] + ([torch.cuda.Stream(device=dev)] if not args.no_pipeline else [])
    ns = len(streams)
    dev_t = [[torch.empty(RES, RES, 4, dtype=torch.float32, device=dev) for _ in range(B)] for _ in range(ns)]
    outs = [[torch.empty_like(dev_t[0][0]) for _ in range(B)] for _ in range(ns)]
    dls = [[torch.empty_like(dev_t[0][0]) for _ in range(B)] for _ in range(ns)]
    losses = [torch.zeros(B, dtype=torch.float32, device=dev) for _ in range(ns)]
    loss_h = [torch.zeros(B, dtype=torch.float32).pin_memory() for _ in range(ns)]
    grads = P.zero_grads(sc)
    copy_stream = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(ns)]
    used = [torch.cuda.Event() for _ in range(ns)]

    def step(i):
        b = i % ns
        st = streams[b]
        vi = [(i * B + j) % n_needed for j in range(B)]
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(used[b])  # the buffers' previous loss reads are done
            for j, v in enumerate(vi):
                dev_t[b][j].copy_(host_t[v % len(host_t)], non_blocking=True)
            copied[b].record(copy_stream)
        if B == 1:
            _, saved = P.render(sc, cams[vi[0]], out=outs[b][0], save=True, stream=st)
        else:
            _, saved = P.render_views([sc] * B, [cams[v] for v in vi], outs=outs[b], save=True, stream=st)
        st.wait_event(copied[b])
        for j in range(B):
            P.l1_loss(outs[b][j], dev_t[b][j], losses[b][j:j + 1], dls[b][j], stream=st)
        used[b].record(st)
        P.render_backward(saved, dls[b], grads, stream=st)
        saved.release()
        with torch.cuda.stream(st):
            loss_h[b].copy_(losses[b], non_blocking=True)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    copy_stream.wait_event(e0)
    for s2 in streams[1:]:
        s2.wait_event(e0)
    for i in range(args.steps):
        step(args.warmup + i)
    for s2 in streams[1:]:
        stream.wait_stream(s2)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), pg, dev)
    return {"value": aggregate_value(world, args.steps, ms, B), "unit": UNIT,
            "h2d_bytes_per_step": B * RES * RES * 4 * 4, "d2h_bytes_per_step": 4 * B,
            "note": f"{B} targets H2D per step on a side stream overlapping the render; steps on "
                    f"{'two streams as the timed loop' if not args.no_pipeline else 'one stream'}"}


# Source files each profiled kernel is built from: a committed DRAM-traffic
# figure is used only while all of them are unchanged.
KERNEL_SOURCES = {
    "raster_bwd": ["raster_bwd.cu", "raster.cuh", "shading.cuh", "ts_common.cuh"],
    "raster_fwd": ["raster_fwd.cu", "raster.cuh", "shading.cuh", "ts_common.cuh"],
}


def kernel_source_hash(kernel: str) -> str:
    import hashlib
    src = os.path.join(ROOT, "paper_2506_13348_b300", "csrc")
    h = hashlib.sha256()
    for fn in KERNEL_SOURCES[kernel]:
        with open(os.path.join(src, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


TRAFFIC_PATH = os.path.join(ROOT, "profiles", "traffic.json")


def read_traffic(kernel: str, views: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current source of that kernel and on launches covering
    `views` views (the bench's views per step); else None."""
    path = TRAFFIC_PATH
    if not os.path.exists(path) or kernel not in KERNEL_SOURCES:
        return None
    with open(path) as f:
        ent = json.load(f).get(kernel)
    if not ent or ent.get("source_sha256") != kernel_source_hash(kernel) or ent.get("views_per_launch") != views:
        return None
    return ent.get("dram_bytes_per_launch")


# Algorithmic bytes of the two rasterisers (per view): what each must move
# at least once.  Both read the pair list (4 B per pair), the first 48 B of
# every visible splat's record (block test and fragment), the last 32 B of
# each splat blended at some pixel, and every distinct texel a blended
# fragment reads (32 B at float32: n_texels_read from the statistics pass).
#   forward: + per pixel rgba 16 and saved state 48 out      -> 64 B / pixel
#   backward: + per pixel dL/dX, dL/dA 48, T and last index 8 in -> 56 B / pixel;
#     texel gradients read and written once per distinct texel (2 x 32 B),
#     record gradients (14 doubles) read and written per blended splat
def raster_bytes(fr, P, texel_bytes=32):
    common = 4 * fr["n_pairs"] + 48 * fr["n_visible"] + 32 * fr["n_items_blended"] + texel_bytes * fr["n_texels_read"]
    return {"raster_fwd": common + 64 * P,
            "raster_bwd": common + 56 * P + 2 * texel_bytes * fr["n_texels_read"] + 2 * 112 * fr["n_items_blended"]}


def stage_bytes(N, K, P, tiles):
    return {"preprocess": 152 * N, "sort_splats": 128 * N, "scan_counts": 20 * N,
            "emit_pairs": 8 * K + 28 * N, "sort_pairs": 40 * K, "tile_ranges": 4 * K + 44 * tiles,
            "shade_bwd": 100 * P, "preprocess_bwd": 192 * N, "l1_loss": 48 * P}


def run_features(args, device):
    """The optional features of the render on the cfg1 step (200k splats,
    8x8 texels, 800x800, forward + L1 + backward): indirect light (per-splat
    SH of degree 2, a random per-pixel visibility in [0, 1]), two-component
    tangent normals, and both, each against the plain step on the same
    scene, cameras and targets."""
    import numpy as np
    import torch

    import paper_2506_13348_b300 as P
    from paper_2506_13348_b300 import _lib
    import scenegen as sg

    dev = torch.device("cuda", device)
    scene, env, cams = build_workload()
    sc = P.Scene.from_arrays(scene, env, device=device)
    n = len(scene["opacity"])
    rng = np.random.default_rng(31)
    sh = torch.from_numpy((rng.normal(size=(n, 9, 3)) * 0.3).astype(np.float32)).to(dev)
    nv = args.feature_steps + 3
    targets = [torch.from_numpy(sg.make_target(i % N_CAMS, RES, RES)).to(dev) for i in range(nv)]
    vis = [torch.from_numpy(rng.uniform(0, 1, size=(RES, RES)).astype(np.float32)).to(dev) for _ in range(nv)]
    out = torch.empty(RES, RES, 4, dtype=torch.float32, device=dev)
    dl = torch.empty_like(out)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)

    def run(indirect, xy):
        sc.upload_indirect(sh if indirect else None)
        sc.set_normal_encoding("xy" if xy else "xyz")
        grads = P.zero_grads(sc)

        def step(i):
            cam = dict(cams[i % N_CAMS], vis=vis[i]) if indirect else cams[i % N_CAMS]
            _, saved = P.render(sc, cam, out=out, save=True)
            P.l1_loss(out, targets[i], loss, dl)
            P.render_backward(saved, dl, grads)
            saved.release()

        for i in range(3):
            step(i)
        torch.cuda.synchronize()
        _lib.profile_enable(True)
        _lib.profile_report()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(args.feature_steps):
            step(3 + i)
        e1.record()
        torch.cuda.synchronize()
        stages = _lib.profile_report()
        _lib.profile_enable(False)
        ms = e0.elapsed_time(e1) / args.feature_steps
        del grads
        return {"ms_per_step": ms, "mpix_per_s": RES * RES / 1e6 / (ms / 1e3),
                "stages_ms": {k: round(v[1] / max(1, v[0]), 4) for k, v in stages.items()
                              if k in ("raster_fwd", "raster_bwd", "shade_bwd")}}

    res = {"workload": "cfg1 step (200k splats, 8x8 texels, 800x800, fwd + L1 + bwd), "
                       f"{args.feature_steps} timed steps per variant",
           "indirect_input": "per-splat SH degree 2 (9 x 3 coefficients, N(0, 0.3)), visibility U[0,1] per pixel"}
    for name, ind, xy in (("plain", False, False), ("indirect", True, False), ("normal_xy", False, True),
                          ("indirect_normal_xy", True, True)):
        res[name] = run(ind, xy)
    for name in ("indirect", "normal_xy", "indirect_normal_xy"):
        res[name]["vs_plain"] = res[name]["ms_per_step"] / res["plain"]["ms_per_step"]
    sc.close()
    torch.cuda.empty_cache()
    return res


def run_hbm_kernels(args, device):
    """The HBM-bound kernels alone: the atlas pack (float32 -> bf16) and one
    Adam step with its bf16 stored copy, on 2^28 float32 values (1 GiB),
    3 warm-up and 10 timed launches each, CUDA events."""
    import torch

    import paper_2506_13348_b300 as P
    from paper_2506_13348_b300 import _lib
    import scenegen as sg

    dev = torch.device("cuda", device)
    n = 1 << 28
    T = 8
    n_splats = n // (T * T * 8)
    geo = sg.make_scene(1, n=n_splats, with_texels=False)
    tex = torch.rand(n, device=dev)
    sc = P.Scene(device)
    sc.upload_gaussians(geo["means"], geo["quats"], geo["scales"], geo["opacity"])
    peaks, peak_kind = load_peaks()
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    out = {"values": n, "peak": f"{hbm:.0f} GB/s ({peak_kind})"}
    _lib.profile_enable(True)
    for i in range(13):
        if i == 3:
            _lib.profile_report()
        _lib.check(_lib.lib().ts_upload_atlas(sc.handle, T, 8, 1, tex.data_ptr(), 1, None), "ts_upload_atlas")
    st = _lib.profile_report()
    pms = st["atlas_pack"][1] / st["atlas_pack"][0]
    out["pack_bf16"] = {"ms": pms, "gb_per_s": n * 6 / (pms / 1e3) / 1e9, "frac": n * 6 / (pms / 1e3) / 1e9 / hbm}
    p, g, m, v = tex, torch.rand(n, device=dev), torch.zeros(n, device=dev), torch.zeros(n, device=dev)
    shadow, _, _ = P.scene_texels(sc)
    for i in range(13):
        if i == 3:
            _lib.profile_report()
        P.adam_update(p, g, m, v, i + 1, 1e-3, shadow_ptr=shadow, shadow_dtype="bf16", zero_grad=False)
    st = _lib.profile_report()
    _lib.profile_enable(False)
    ams = st["adam"][1] / st["adam"][0]
    # p g m v in, p m v out, the bf16 copy out (the gradient is kept here)
    ab = n * (16 + 12 + 2)
    out["adam_bf16_shadow"] = {"ms": ams, "gb_per_s": ab / (ams / 1e3) / 1e9, "frac": ab / (ams / 1e3) / 1e9 / hbm}
    sc.close()
    return out


def run_packing_probe(args, device):
    """One 800x800 forward of the 200k-splat scene (8x8 FP32 texels) through
    the hardware-texture atlas for each chart packing: splat-id order, then the
    Morton order of the splat centres (two k_raster_fwd launches for a
    profiler to compare texture-cache hit rates)."""
    import torch

    import paper_2506_13348_b300 as P
    import scenegen as sg

    dev = torch.device("cuda", device)
    scene, env, cams = build_workload()
    sc = P.Scene.from_arrays(scene, env, device=device)
    img = torch.empty(RES, RES, 4, device=dev)
    out = {}
    for packing in ("splat_id", "morton"):
        sc.build_atlas2d("f32", packing=packing)
        sc.set_sampler("hw_atlas")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        P.render(sc, cams[5], out=img)
        e1.record()
        torch.cuda.synchronize()
        out[packing] = {"ms": e0.elapsed_time(e1)}
    sc.close()
    return out


def run_sampling(args, device):
    """The shape of the paper's Table 3: forward-render throughput of textured
    splats relative to the same splats without textures, for T = 2, 4, 8, 16,
    with the software bilinear filter (FP32 charts) and with the hardware
    texture units (FP32 2-D atlases, tex2D).  Geometry, environment and
    cameras of the 200k-splat 800x800 workload; the untextured baseline
    renders one attribute vector per splat (flat sampler, T = 1).  The
    hardware path is timed with charts in splat id order (the paper's) and in
    the Morton order of the splat centres.  Each figure is views per second
    over the same views.  The training step (forward with saved state, L1,
    backward) is timed per T too, against T = 1 (one texel per splat: the
    per-splat attribute model through the same software path)."""
    import torch

    import paper_2506_13348_b300 as P
    import scenegen as sg

    dev = torch.device("cuda", device)
    geo = sg.make_scene(1, with_texels=False)
    env = sg.make_env(1, cube_res=32, levels=1, irr_res=8, lut_res=128)
    cams = sg.fibonacci_cameras(N_CAMS, 4.0, RES, RES)
    nv = max(4, args.sampling_views)
    img = torch.empty(RES, RES, 4, device=dev)

    def fps(sc):
        for i in range(3):
            P.render(sc, cams[i], out=img)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(nv):
            P.render(sc, cams[i % N_CAMS], out=img)
        e1.record()
        torch.cuda.synchronize()
        return nv / (e0.elapsed_time(e1) / 1e3)

    tgt = torch.from_numpy(sg.make_target(0, RES, RES)).to(dev)
    dl = torch.empty_like(img)
    loss = torch.zeros(1, device=dev)

    def train_ms(sc):
        grads = P.zero_grads(sc)

        def step(i):
            _, saved = P.render(sc, cams[i % N_CAMS], out=img, save=True)
            P.l1_loss(img, tgt, loss, dl)
            P.render_backward(saved, dl, grads)
            saved.release()

        for i in range(3):
            step(i)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(nv // 2):
            step(i)
        e1.record()
        torch.cuda.synchronize()
        del grads
        return e0.elapsed_time(e1) / (nv // 2)

    def scene_with(T):
        sc = P.Scene(device)
        sc.upload_gaussians(geo["means"], geo["quats"], geo["scales"], geo["opacity"])
        sc.upload_atlas(sg.scenes.texels_torch(len(geo["opacity"]), T, seed=1, device=dev), "f32")
        sc.upload_envmap(env, "f32")
        return sc

    sc = scene_with(1)
    base_train = train_ms(sc)
    sc.set_sampler("flat")
    base = fps(sc)
    sc.close()
    out = {"workload": "200k splats (cfg1 geometry), 800x800, forward render, views/s over "
                       f"{nv} views; FP32 charts (software) vs FP32 2-D atlases (tex2D)",
           "untextured_fps": base, "train_ms_T1": base_train,
           "paper_table3_ratios": {"software": [0.90, 0.86, 0.85, 0.79], "hardware": [0.92, 0.93, 0.94, 0.91]}}
    for T in (2, 4, 8, 16):
        sc = scene_with(T)
        sw = fps(sc)
        tr = train_ms(sc)
        P.render(sc, cams[0], out=img)
        ref = img.clone()
        sc.build_atlas2d("f32")
        sc.set_sampler("hw_atlas")
        hw = fps(sc)
        P.render(sc, cams[0], out=img)
        d = (img - ref).abs()[..., :3]
        sc.build_atlas2d("f32", packing="morton")
        hw_m = fps(sc)
        sc.close()
        torch.cuda.empty_cache()
        out[f"T{T}"] = {"software_fps": sw, "hardware_fps": hw, "hardware_morton_fps": hw_m,
                        "train_ms": tr, "train_ratio": base_train / tr,
                        "software_ratio": sw / base, "hardware_ratio": hw / base, "hardware_morton_ratio": hw_m / base,
                        "hw_vs_software_rgb": {"max_abs": float(d.max()), "mean_abs": float(d.mean())}}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if (args.serve_only or args.large_only or args.precision_only or args.sampling_only or args.features_only
            or args.hbm_kernels_only or args.packing_probe):
        import torch
        torch.cuda.set_device(dist_env()[2])
        res = {}
        if args.serve_only:
            res["serving"] = run_serving(args, dist_env()[2])
        if args.large_only:
            res["large_scene"] = run_large_scene(args, dist_env()[2])
        if args.precision_only:
            res["precision"] = run_precision(args, dist_env()[2])
            inp = res["precision"].pop("_oracle_inputs")
            if not args.no_cpu_baseline:
                res["precision"]["vs_fp64_oracle"] = precision_vs_oracle(inp)
        if args.sampling_only:
            res["texture_sampling"] = run_sampling(args, dist_env()[2])
        if args.features_only:
            res["features"] = run_features(args, dist_env()[2])
        if args.hbm_kernels_only:
            res["hbm_kernels"] = run_hbm_kernels(args, dist_env()[2])
        if args.packing_probe:
            res["packing_probe"] = run_packing_probe(args, dist_env()[2])
        print(json.dumps(res))
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
