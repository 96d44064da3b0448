#!/usr/bin/env python
"""Benchmark of the fisheye plane-sweep + TSDF fusion hot path.

Workload (one step = one synchronised frame through the whole path): the
street rig, reference + 2 matching fisheye cameras at 1280x1024 (unified
model, xi ~ U[0.8, 1.2], radial-tangential distortion), seeded street scene
rendered synthetically; multi-resolution sweep (320x256 with 64
fronto-parallel + 32 ground-parallel planes and a 7x7 ZNCC window; central
640x512 crop at full resolution with 128 planes and a 9x9 window), box
masks, and fusion into a voxel-block TSDF (8^3 blocks, 10 cm voxels,
0.5 m truncation, 60 x 3 x 60 m local map) along the straight 1 m/frame
trajectory.

Metric: depth+TSDF frames/s (whole job, all ranks), with the plane-sweep
rate in Gpix.planes/s beside it.  Each rank runs an independent sequence
(seed + rank): no data-path collective, weak scaling.

  python bench.py [--gpus N] [--steps K] [--warmup W]          # CUDA path
  python bench.py --impl reference [--steps K] [--warmup W]    # the FP64 CPU oracle
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "plane-sweep Gpix·planes/s and depth+TSDF frames/s on 1 GB300 vs plain FP32 form"
UNIT = "frames/s"
# algorithmic FP32 operations per (reference pixel, plane, matching camera):
# warp 64 (plane intersection 4, rigid transform 18, unified projection 12,
# distortion 18, bilinear sample 12), window statistics 18 (w^2 and r w
# products, running horizontal + vertical sums of 4 quantities), ZNCC cost 9,
# camera minimum 1
FLOP_PER_UNIT = 92
# TSDF integration: each voxel of a listed block is read and written once ({D, w} float32 pairs)
BYTES_PER_VOXEL = 16
# dram__bytes_read.sum + dram__bytes_write.sum of one sweep_kernel launch on the street frame (FP32 images),
# from an ncu capture of the current kernel (28,467,712 B read + 12,621,824 B written)
SWEEP_DRAM_BYTES_STREET = 41_089_536


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--config", choices=["street", "tiny", "ring", "ringloop", "batch", "diff", "cpubase"],
                    default="street",
                    help="street: the paper-shaped frame (default); tiny: 160x128, 1 matching camera, 32 planes, "
                         "dense 64^3 TSDF; ring: 4 cameras, 256 full-resolution planes, "
                         "2 cm voxels on a 500 m loop; batch: 64 uneven sweeps in one persistent launch; "
                         "diff: soft-argmin forward/backward and extrinsic refinement; ringloop: fusion of the "
                         "whole 1000-frame ring at 2 cm")
    ap.add_argument("--batch-size", type=int, default=64, help="sweeps per batch (--config batch)")
    ap.add_argument("--half", action="store_true", help="FP16 storage of the matching images")
    ap.add_argument("--sweep-depth", action="store_true",
                    help="--config ringloop: fuse the sweep's own depth maps (a contiguous stretch of the loop, "
                         "sweep + fusion timed) instead of the renderer's true ranges")
    ap.add_argument("--shard", action="store_true",
                    help="N > 1: one sequence split over the ranks (each rank sweeps a plane range of every frame, "
                         "one all-gather of the per-pixel records, every rank merges; the TSDF as hash parts), "
                         "strong scaling, instead of independent sequences")
    return ap.parse_args()


def workload(args, seed):
    import scenes
    if args.config == "ring":
        return scenes.ring(seed, n_frames=1000)
    if args.config == "tiny":
        return scenes.tiny(seed, n_frames=100)
    return scenes.street(seed, n_frames=100)


def workload_config(args, wl, nf, world):
    """The `config` object of a street / ring line (the same for both arms)."""
    levels = {"street": "320x256 (64 fronto + 32 ground, 7x7) + 640x512 crop (128 fronto, 9x9)",
              "tiny": "160x128 (32 fronto on 0.5-20 m, 5x5)"}
    tsdf = {"street": "8^3 blocks, 0.1 m voxels, mu 0.5 m, 60x3x60 m local map",
            "tiny": "dense 64^3 grid, 0.05 m voxels, mu 0.2 m"}
    return {"workload": wl.name, "ref": f"{wl.rig.ref.width}x{wl.rig.ref.height}",
            "matching_cams": len(wl.rig.cams),
            "levels": levels.get(args.config, "1280x1024 (256 fronto, 9x9)"),
            "tsdf": tsdf.get(args.config, "8^3 blocks, 0.02 m voxels, mu 0.1 m, 60x3x60 m local map, "
                                          "2^23-block pool"),
            "image_storage": "fp16" if getattr(args, "half", False) else "fp32", "frames": nf,
            "l2": "flushed between steps (256 MB write outside the step events)",
            "parallelism": f"replicas x{world} (independent sequences)"}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(values, device="cpu"):
    """Each value's maximum over the ranks of the job (the job ends when its
    slowest rank does); the values themselves when there is one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def rank_seed(seed: int, rank: int) -> int:
    """Seed of a rank's independent sequence (replicas: no data exchange)."""
    return seed + rank


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ----------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self):
        return time.time()

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0=None, t1=None):
        sm, mx, reasons = [], [], set()
        for ts, line in self.lines:
            if t0 is not None and not (t0 <= ts <= t1 + 0.06):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- CPU oracle leg

def oracle_band(wl, imgs, band: int, n_bands: int, outs):
    """Oracle sweep of the rows y = band (mod n_bands) of every level of one
    frame (every pixel of those rows; interleaved, so that each band holds a
    like share of sky, ground and facades), written into outs[level]
    (dicts of full level arrays)."""
    import oracle
    for lv, o in zip(wl.levels, outs):
        H, W = oracle.level_shape(wl.rig, lv)
        rows = np.arange(band, H, n_bands)
        yy, xx = np.meshgrid(rows, np.arange(W), indexing="ij")
        pix = np.stack([xx.ravel(), yy.ravel()], axis=1).astype(np.int32)
        r = oracle.sweep_level(wl.rig, lv, imgs, pix=pix)
        for k in ("depth", "c1", "c2", "kstar"):
            o[k][rows] = r[k].reshape(len(rows), W)


def oracle_level_outs(wl):
    import oracle
    outs = []
    for lv in wl.levels:
        H, W = oracle.level_shape(wl.rig, lv)
        outs.append({"depth": np.zeros((H, W)), "c1": np.zeros((H, W)), "c2": np.zeros((H, W)),
                     "kstar": np.zeros((H, W), np.int32)})
    return outs


def oracle_finish_frame(wl, f, outs, T):
    """Merge of the oracle's level maps, boxes, and fusion of the merged map."""
    import oracle
    low = crop = None
    s, cw, ch = 1, 0, 0
    for lv, o in zip(wl.levels, outs):
        if lv.kind == 0:
            low, s = o["depth"], lv.factor
        else:
            crop, cw, ch = o["depth"], lv.crop_w, lv.crop_h
    D = oracle.merge(wl.rig.ref.width, wl.rig.ref.height, low, s, crop, cw, ch, wl.boxes[f])
    T.integrate(D.astype(np.float32), wl.rig.ref, wl.world_to_ref[f], wl.local_center(f))


def oracle_frame_s(wl, imgs, f, threads, n_bands=1, bands=None):
    """Seconds of the oracle's whole path for frame f on `threads` threads:
    the sweep of both levels at every pixel (or only `bands` of n_bands
    interleaved row bands, then scaled by n_bands / len(bands)), the merge,
    the boxes and the fusion of the frame's merged map into a fresh map."""
    import oracle
    oracle.set_threads(threads)
    outs = oracle_level_outs(wl)
    bands = list(range(n_bands)) if bands is None else list(bands)
    t0 = time.perf_counter()
    for b in bands:
        oracle_band(wl, imgs, b, n_bands, outs)
    t_sweep = (time.perf_counter() - t0) * n_bands / len(bands)
    T = oracle.Tsdf(wl.tsdf)
    t1 = time.perf_counter()
    oracle_finish_frame(wl, f, outs, T)
    return t_sweep + time.perf_counter() - t1, t_sweep


def cpu_baseline(wl, frames, tiny_wl=None):
    """Frames/s of the FP64 oracle on the host cores, measured: frame 0 of the
    workload through the whole path on every core (nproc threads), the same
    frame on one thread over every 16th row of each level (scaled to the
    frame) plus its full fusion, and, with tiny_wl, the tiny workload's
    frame on one thread and on every core."""
    import oracle
    n = os.cpu_count() or 1
    imgs = frames[0][0]
    t_all, sw_all = oracle_frame_s(wl, imgs, 0, n)
    t_one, sw_one = oracle_frame_s(wl, imgs, 0, 1, n_bands=16, bands=[7])
    out = {"value": 1.0 / t_all, "unit": UNIT, "cores": n, "threads": oracle.set_threads(n), "kind": "oracle",
           "sample": f"frame 0 of {wl.name}: both levels swept at every pixel, merge, boxes and fusion of the "
                     f"merged map, on {n} threads ({t_all:.1f} s)",
           "sweep_s_per_frame": sw_all,
           "single_thread": {"value": 1.0 / t_one, "unit": UNIT, "threads": 1,
                             "sample": "frame 0, every 16th row of each level (rows 7 mod 16) swept on one thread "
                                       "and scaled x16, plus the frame's merge and fusion",
                             "sweep_s_per_frame": sw_one}}
    if tiny_wl is not None:
        import scenes
        timgs, _ = scenes.FrameSource(tiny_wl).frame(0)
        timgs = [i.numpy() for i in timgs]
        a, _ = oracle_frame_s(tiny_wl, timgs, 0, 1)
        b, _ = oracle_frame_s(tiny_wl, timgs, 0, n)
        out["tiny"] = {"workload": tiny_wl.name, "frames": tiny_wl.n_frames, "single_thread": 1.0 / a,
                       f"threads_{n}": 1.0 / b, "unit": UNIT}
    oracle.set_threads(n)
    return out


# ----------------------------------------------------------------- main

def render_frames(wl, n, device):
    import scenes
    src = scenes.FrameSource(wl, device=device)
    out = []
    for f in range(n):
        imgs, rng = src.frame(f, with_range=True)
        d = rng.numpy().astype(np.float32)
        H, W = d.shape
        for x0, y0, x1, y1 in wl.boxes[f]:
            d[max(0, y0):min(H, y1), max(0, x0):min(W, x1)] = 0
        out.append(([i.numpy() for i in imgs], d))
    return out


def run_reference(args):
    """The FP64 oracle as it stands, on every host core, through the whole
    path: each step sweeps one interleaved row band (every 4th row of both
    levels) of the current frame at every pixel; the step that completes a
    frame also merges its levels, applies the boxes and fuses the merged
    map.  Four steps make a frame, so the K timed steps measure K/4 whole
    frames; value = frames / seconds, ms_per_step = the measured mean step."""
    import scenes
    import oracle
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    n_bands = 4
    wl = workload(args, args.seed)
    n = args.warmup + args.steps
    nf = (n + n_bands - 1) // n_bands
    try:
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
    except Exception:
        dev = "cpu"
    frames = render_frames(wl, nf, dev)   # input synthesis only (torch ops)
    threads = oracle.set_threads(os.cpu_count() or 1)
    T = oracle.Tsdf(wl.tsdf)
    outs = oracle_level_outs(wl)
    times = []
    for i in range(n):
        f, b = i // n_bands, i % n_bands
        t0 = time.perf_counter()
        oracle_band(wl, frames[f][0], b, n_bands, outs)
        if b == n_bands - 1:
            oracle_finish_frame(wl, f, outs, T)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    val = (len(times) / n_bands) / total
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / len(times) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, wl, nf, world),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": os.cpu_count() or 1, "threads": threads,
                             "kind": "oracle",
                             "sample": f"each step: one of {n_bands} row bands of both levels swept at every pixel; "
                                       f"every {n_bands}th step also merges, masks and fuses the frame; "
                                       f"{len(times) / n_bands:.2f} frames timed"},
            "step_ms": {"median": statistics.median(times) * 1e3, "min": min(times) * 1e3, "max": max(times) * 1e3},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    import scenes
    import paper_1809_06132_gb300 as P

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks, peaks_src = load_peaks()

    wl = workload(args, rank_seed(args.seed, rank))
    n_total = args.warmup + args.steps
    nf = min(n_total, 40 if args.config == "ring" else 100)
    t_r = time.time()
    frames = render_frames(wl, nf, f"cuda:{local}")
    render_s = time.time() - t_r
    imgs_dev = [[torch.from_numpy(i).to(dev) for i in imgs] for imgs, _ in frames]
    imgs_host = [[torch.from_numpy(i).pin_memory() for i in imgs] for imgs, _ in frames]
    H, W = wl.rig.ref.height, wl.rig.ref.width
    stream = torch.cuda.current_stream()

    sw = P.Sweep(wl.rig, wl.levels, image_half=args.half)
    T = P.Tsdf(wl.tsdf, wl.rig.ref)
    depth = torch.empty((H, W), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def step(i):
        f = i % nf
        sw.depth(imgs_dev[f], boxes=wl.boxes[f], out=depth, stream=stream)
        T.integrate(depth, wl.world_to_ref[f], wl.local_center(f), stream=stream)

    for i in range(args.warmup):
        step(i)
    assert T.status(stream) == P.PS_OK
    sw.profile(args.steps)
    T.profile(args.steps)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step(args.warmup + k)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    if world > 1:
        dist.barrier()
    step_ms = sorted(a.elapsed_time(b) for a, b in ev)
    ms = sum(step_ms)
    sweep_ms, n_sw = sw.profile_read()
    tsdf_ms, n_ts = T.profile_read()
    st = T.status(stream)
    ms = max_over_ranks([ms], dev)[0]
    ms_per_step = ms / args.steps
    value = world * args.steps / (ms / 1e3)
    n_blocks = T.count(stream)
    n_listed = T.listed(stream)  # the last timed frame's visible-block list
    # rays the allocation stage walks per frame: pixels with a depth in the
    # merged, masked maps of the timed frames (counted after the timing)
    rays = []
    for k in range(min(args.steps, nf)):
        f = (args.warmup + k) % nf
        sw.depth(imgs_dev[f], boxes=wl.boxes[f], out=depth, stream=stream)
        rays.append(int((depth > 0).sum().item()))
    rays_per_frame = statistics.mean(rays)

    # e2e: host images -> device -> depth + fusion -> depth map back to host, per step
    sw.profile(0)
    T.profile(0)
    T2 = P.Tsdf(wl.tsdf, wl.rig.ref)
    host_depth = torch.empty((H, W), dtype=torch.float32).pin_memory()

    def step_host(i):
        f = i % nf
        sw.frame_host(imgs_host[f], boxes=wl.boxes[f], tsdf=T2, world_to_ref=wl.world_to_ref[f],
                      local_center=wl.local_center(f), depth_out=host_depth, stream=stream)

    for i in range(args.warmup):
        step_host(i)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        ts = time.perf_counter()
        step_host(args.warmup + k)
        e2e_ms += (time.perf_counter() - ts) * 1e3
    # the same through the frame pipeline (copy-in / compute: sweep then fusion / copy-out
    # streams, two frames in flight): K pushes and the final flush, host images in, depth maps out
    T3 = P.Tsdf(wl.tsdf, wl.rig.ref)
    pipe = P.Pipeline(sw, T3)
    host_outs = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(2)]

    def push(i):
        f = i % nf
        pipe.push(imgs_host[f], boxes=wl.boxes[f], world_to_ref=wl.world_to_ref[f],
                  local_center=wl.local_center(f), depth_out=host_outs[i & 1])

    for i in range(args.warmup):
        push(i)
    pipe.flush()
    flush.zero_()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ts = time.perf_counter()
    for k in range(args.steps):
        push(args.warmup + k)
    pipe.flush()
    pipe_ms = (time.perf_counter() - ts) * 1e3
    assert T3.status() == P.PS_OK
    pipe.close()
    e2e_ms, pipe_ms = max_over_ranks([e2e_ms, pipe_ms], dev)
    clocks.stop()
    clk = clocks.summary(t0, t1)
    if not clk.get("samples"):
        clk = clocks.summary()
    h2d = H * W + sum(c.width * c.height for c in wl.rig.cams)
    d2h = 4 * H * W

    pix_planes = wl.pix_planes()
    units = sum(w * h * lv.n_planes * len(wl.rig.cams)
                for lv, (h, w) in zip(wl.levels, sw.level_shapes()))
    k_ms = sweep_ms[1] / max(1, n_sw)
    depth_ms = sum(sweep_ms) / max(1, n_sw)
    sm_max = clk.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tflops = n_sm * 128 * 2 * float(sm_max) * 1e6 / 1e12
    achieved = units * FLOP_PER_UNIT / (k_ms * 1e-3) / 1e12
    integ_ms = tsdf_ms[3] / max(1, n_ts)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args, wl, nf, world),
        "step_ms": {"median": statistics.median(step_ms), "p10": float(np.percentile(step_ms, 10)),
                    "p90": float(np.percentile(step_ms, 90)), "mean": ms_per_step,
                    "source": "CUDA events around each step on the launching stream (rank 0)"},
        "sweep": {"value": pix_planes / (depth_ms * 1e-3) / 1e9, "unit": "Gpix·planes/s",
                  "kernel_only": pix_planes / (k_ms * 1e-3) / 1e9,
                  "gpix_plane_cam_per_s": units / (k_ms * 1e-3) / 1e9,
                  "pix_planes_per_frame": pix_planes, "ms_depth_stage": depth_ms, "ms_sweep_kernel": k_ms},
        "tsdf": {"ms_per_frame": sum(tsdf_ms) / max(1, n_ts),
                 "ms_stages": {"depth_max": tsdf_ms[0] / max(1, n_ts), "alloc": tsdf_ms[1] / max(1, n_ts),
                               "visible": tsdf_ms[2] / max(1, n_ts), "integrate": integ_ms},
                 "blocks_allocated": n_blocks, "status": st,
                 "integrate_bw": {"listed_blocks": n_listed,
                                  "gbs": n_listed * 512 * BYTES_PER_VOXEL / (integ_ms * 1e-3) / 1e9 if integ_ms else None,
                                  "note": "16 B per voxel of the last timed frame's listed blocks over the mean "
                                          "integrate time per frame (the listed count varies little between frames)"},
                 "alloc": {"rays_per_frame": rays_per_frame,
                           "rays_per_s": rays_per_frame / (tsdf_ms[1] / max(1, n_ts) * 1e-3),
                           "note": "segments [d - mu, d + mu] walked by the allocation stage per second"}},
        "roofline": {"kernel": "sweep_kernel", "bound": "alu", "achieved": achieved, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                     "traffic": SWEEP_DRAM_BYTES_STREET if args.config == "street" and not args.half else None,
                     "peak_source": f"{n_sm} SMs x 128 FP32 lanes x 2 (FMA) x {sm_max:.0f} MHz "
                                    f"(max SM clock, {'sampled' if clk.get('sm_max_mhz') else 'recipe'})",
                     "flop_per_unit": FLOP_PER_UNIT, "units_per_launch": units},
        "e2e": {"value": world * args.steps / (pipe_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "api": "ps_pipe_push x K + ps_pipe_flush (two frames in flight)",
                "serial": world * args.steps / (e2e_ms / 1e3), "serial_api": "psweep_frame_host per frame"},
        # one prep launch for every level (reference images, statistics, quads), the sweep, the merge; 4 TSDF stages
        "gpu_launches": args.steps * (1 + 2 + 4),
        "clocks": clk,
        "render_s": render_s,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.config in ("street", "tiny"):
        import scenes
        line["cpu_baseline"] = cpu_baseline(wl, frames, scenes.tiny(args.seed) if args.config == "street" else None)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """64 uneven sweeps (image sizes 256x200 .. 1024x768, 32 .. 256 planes, 1 .. 4
    matching cameras) per step: autotune the batch options, then time the
    batch as one persistent launch replayed from a CUDA graph, against the
    same sweeps as 64 single-frame calls.  Per-sweep latency = device clock
    from the kernel start to the sweep's finished depth map."""
    import torch
    import torch.distributed as dist

    import scenes
    import paper_1809_06132_gb300 as P

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wls = scenes.batch_mix(rank_seed(args.seed, rank), n=args.batch_size)
    t_r = time.time()
    images, boxes, host_imgs = [], [], []
    for wl in wls:
        imgs, _ = scenes.FrameSource(wl, device=f"cuda:{local}").frame(0)
        host_imgs.append([torch.from_numpy(np.ascontiguousarray(i.numpy())).pin_memory() for i in imgs])
        images.append([h.to(dev) for h in host_imgs[-1]])
        boxes.append(wls[len(boxes)].boxes[0])
    render_s = time.time() - t_r
    sweeps = [P.Sweep(wl.rig, wl.levels) for wl in wls]
    outs = [torch.empty((wl.rig.ref.height, wl.rig.ref.width), dtype=torch.float32, device=dev) for wl in wls]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    pix_planes = sum(wl.pix_planes() for wl in wls)
    units = sum(wl.pix_planes() * len(wl.rig.cams) for wl in wls)

    # autotuner: tile height x planes per pass x plane chunk
    cands = [P.batch_opts(tile_h=t, kp=k, plane_chunk=c) for t in (16, 24) for k in (1, 2) for c in (16, 32, 64)]
    with torch.cuda.stream(stream):
        best, tune_ms = P.batch_autotune(sweeps, images, cands, boxes=boxes, outs=outs, reps=3, stream=stream)
    o = cands[best]
    tuned = dict(tile_h=o.tile_h, kp=o.kp, plane_chunk=o.plane_chunk)
    o.use_graph = 1
    B = P.Batch(sweeps, opts=o)

    def timed(fn, k_steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k_steps)]
        lat = []
        for k in range(k_steps):
            flush.zero_()
            torch.cuda.current_stream().synchronize()
            ev[k][0].record(stream)
            fn()
            ev[k][1].record(stream)
            stream.synchronize()
            if fn is run_batch_once:
                lat.append(B.timing()[0])
        return [a.elapsed_time(b) for a, b in ev], lat

    def run_batch_once():
        B.run(images, boxes=boxes, outs=outs, stream=stream)

    def run_singles():
        for sw, im, bx, out in zip(sweeps, images, boxes, outs):
            sw.depth(im, boxes=bx, out=out, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            run_batch_once()
        stream.synchronize()
        assert B.status() == P.PS_OK
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.3)
        if world > 1:
            dist.barrier()
        t0 = time.time()
        ms, lat = timed(run_batch_once, args.steps)
        t1 = time.time()
        for _ in range(args.warmup):
            run_singles()
        ms_single, _ = timed(run_singles, max(3, args.steps // 4))
        # the same batch without the graph (four API calls per run)
        Bg = P.Batch(sweeps, opts=P.batch_opts(tile_h=o.tile_h, kp=o.kp, plane_chunk=o.plane_chunk))
        for _ in range(2):
            Bg.run(images, boxes=boxes, outs=outs, stream=stream)
        ms_nograph = []
        for k in range(max(3, args.steps // 4)):
            flush.zero_()
            stream.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            Bg.run(images, boxes=boxes, outs=outs, stream=stream)
            b.record(stream)
            stream.synchronize()
            ms_nograph.append(a.elapsed_time(b))
        # end to end: pinned host images in, every depth map out, per step
        host_out = [torch.empty(o_.shape, dtype=torch.float32).pin_memory() for o_ in outs]
        e2e = []
        for k in range(max(3, args.steps // 4)):
            flush.zero_()
            torch.cuda.synchronize()
            ts = time.perf_counter()
            for hs, ds in zip(host_imgs, images):
                for h_, d_ in zip(hs, ds):
                    d_.copy_(h_, non_blocking=True)
            B.run(images, boxes=boxes, outs=outs, stream=stream)
            for d_, h_ in zip(outs, host_out):
                h_.copy_(d_, non_blocking=True)
            stream.synchronize()
            e2e.append(time.perf_counter() - ts)
    # many small sweeps: where one launch pays most
    small = scenes.batch_mix(rank_seed(args.seed, rank) + 100, n=args.batch_size, sizes=((256, 200), (320, 256)),
                             planes=(32, 64))
    s_sweeps, s_imgs, s_boxes = [], [], []
    for w in small:
        im, _ = scenes.FrameSource(w, device=f"cuda:{local}").frame(0)
        s_imgs.append([torch.from_numpy(np.ascontiguousarray(x.numpy())).to(dev) for x in im])
        s_sweeps.append(P.Sweep(w.rig, w.levels))
        s_boxes.append(w.boxes[0])
    s_outs = [torch.empty((w.rig.ref.height, w.rig.ref.width), dtype=torch.float32, device=dev) for w in small]
    with torch.cuda.stream(stream):
        Bs = P.Batch(s_sweeps, opts=P.batch_opts(tile_h=o.tile_h, kp=o.kp, plane_chunk=o.plane_chunk, use_graph=True))

        def small_batch():
            Bs.run(s_imgs, boxes=s_boxes, outs=s_outs, stream=stream)

        def small_singles():
            for sw_, im_, bx_, out_ in zip(s_sweeps, s_imgs, s_boxes, s_outs):
                sw_.depth(im_, boxes=bx_, out=out_, stream=stream)

        for _ in range(args.warmup):
            small_batch()
            small_singles()
        sb, sl = [], []
        for k in range(max(3, args.steps // 2)):
            for fn, acc in ((small_batch, sb), (small_singles, sl)):
                flush.zero_()
                stream.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                stream.synchronize()
                acc.append(a.elapsed_time(b))
        small_lat = sorted(Bs.timing()[0])
    small_pp = sum(w.pix_planes() for w in small)
    # queue order: the same 64 sweeps queued shortest first, as drawn, largest
    # first, and largest / smallest alternating (given order of a permutation)
    work = [wl.pix_planes() * len(wl.rig.cams) for wl in wls]
    by_size = sorted(range(len(wls)), key=lambda i: work[i])
    alt = [x for pair in zip(reversed(by_size), by_size) for x in pair][:len(wls)]
    seen, interleaved = set(), []
    for i in alt:
        if i not in seen:
            seen.add(i)
            interleaved.append(i)
    orders = {"shortest_first": (list(range(len(wls))), P.BATCH_SHORTEST_FIRST),
              "as_drawn": (list(range(len(wls))), P.BATCH_GIVEN_ORDER),
              "largest_first": (list(reversed(by_size)), P.BATCH_GIVEN_ORDER),
              "large_small_interleaved": (interleaved, P.BATCH_GIVEN_ORDER)}
    order_cmp = {}
    with torch.cuda.stream(stream):
        for name, (perm, mode) in orders.items():
            Bo = P.Batch([sweeps[i] for i in perm], opts=P.batch_opts(tile_h=o.tile_h, kp=o.kp,
                                                                    plane_chunk=o.plane_chunk, order=mode))
            args_o = ([images[i] for i in perm], [boxes[i] for i in perm], [outs[i] for i in perm])
            for _ in range(2):
                Bo.run(args_o[0], boxes=args_o[1], outs=args_o[2], stream=stream)
            ms_o, lat_o = [], []
            for _ in range(max(3, args.steps // 2)):
                flush.zero_()
                stream.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                Bo.run(args_o[0], boxes=args_o[1], outs=args_o[2], stream=stream)
                b.record(stream)
                stream.synchronize()
                ms_o.append(a.elapsed_time(b))
                lat_o.extend(Bo.timing()[0])
            lat_o.sort()
            order_cmp[name] = {"batch_ms": statistics.median(ms_o),
                               "gpix_planes_s": pix_planes / (statistics.median(ms_o) * 1e-3) / 1e9,
                               "latency_p50_ms": lat_o[len(lat_o) // 2],
                               "latency_p99_ms": lat_o[min(len(lat_o) - 1, int(0.99 * len(lat_o)))]}
            Bo.close()
    clocks.stop()
    clk = clocks.summary(t0, t1)
    if not clk.get("samples"):
        clk = clocks.summary()
    batch_ms = max_over_ranks([statistics.median(ms)], dev)[0]
    all_lat = sorted(x for step in lat for x in step)
    pct = lambda q: all_lat[min(len(all_lat) - 1, int(q * len(all_lat)))]  # noqa: E731
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak_tflops = n_sm * 128 * 2 * float(sm_max) * 1e6 / 1e12
    achieved = units * FLOP_PER_UNIT / (batch_ms * 1e-3) / 1e12
    h2d = sum(int(h.numel()) for hs in host_imgs for h in hs)
    d2h = sum(4 * int(o_.numel()) for o_ in outs)
    line = {
        "metric": "batched plane-sweep Gpix·planes/s (uneven sweeps, one persistent launch)",
        "value": world * pix_planes / (batch_ms * 1e-3) / 1e9, "unit": "Gpix·planes/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": batch_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch-mix-{len(wls)}", "sizes": "256x200 / 320x256 / 640x512 / 1024x768",
                   "planes": "32 / 64 / 128 / 256 fronto, 7x7", "matching_cams": "1-4",
                   "pix_planes_per_batch": pix_planes, "tuned": tuned, "graph": True,
                   "l2": "flushed between steps (256 MB write outside the step events)"},
        "latency_ms": {"p50": pct(0.5), "p99": pct(0.99), "max": all_lat[-1], "span_median": batch_ms,
                       "source": "device global timer, kernel start to each sweep's finished depth map"},
        "compare": {"singles_ms": statistics.median(ms_single), "batch_no_graph_ms": statistics.median(ms_nograph),
                    "speedup_vs_singles": statistics.median(ms_single) / batch_ms},
        "small_mix": {"sweeps": len(small), "sizes": "256x200 / 320x256", "planes": "32 / 64",
                      "pix_planes_per_batch": small_pp, "batch_ms": statistics.median(sb),
                      "singles_ms": statistics.median(sl), "speedup_vs_singles": statistics.median(sl) /
                      statistics.median(sb), "gpix_planes_s": small_pp / (statistics.median(sb) * 1e-3) / 1e9,
                      "latency_ms": {"p50": small_lat[len(small_lat) // 2], "p99": small_lat[-1]}},
        "queue_order": order_cmp,
        "autotune": [{"tile_h": c.tile_h, "kp": c.kp, "plane_chunk": c.plane_chunk, "ms": m}
                     for c, m in zip(cands, tune_ms)],
        "roofline": {"kernel": "batch_kernel", "bound": "alu", "achieved": achieved, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": None,
                     "flop_per_unit": FLOP_PER_UNIT, "units_per_launch": units},
        "e2e": {"value": world * pix_planes / statistics.median(e2e) / 1e9, "unit": "Gpix·planes/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps, "clocks": clk, "render_s": render_s,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_diff(args):
    """Differentiable sweep: forward and backward time of the soft-argmin
    depth on the 96x80 rig (2 matching cameras, 32 planes, 5x5) and on a
    640x512 rig (2 cameras, 128 planes), and a 50-step extrinsic refinement
    from a 0.5 degree / 2 cm perturbation on the 192x160 rig."""
    import torch

    import scenes
    import paper_1809_06132_gb300 as P
    from paper_1809_06132_gb300.refine import refine_extrinsic
    from scenes.configs import Rig

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = {}
    for name, kw in (("diff-96x80-2cam-32planes", dict(width=96, height=80, n_planes=32)),
                     ("diff-640x512-2cam-128planes", dict(width=640, height=512, n_planes=128))):
        wl = scenes.diff(args.seed, **kw)
        imgs, _ = scenes.FrameSource(wl, device=f"cuda:{local}").frame(0)
        ims = [torch.from_numpy(i.numpy().astype(np.float32) / 255.0).to(dev) for i in imgs]
        sw = P.SoftSweep(wl.rig, wl.levels[0])
        g = torch.ones((wl.rig.ref.height, wl.rig.ref.width), dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            r, c, aux = sw.forward(ims)
            sw.backward(ims, None, aux, g, g)
        tf, tb = [], []
        for _ in range(args.steps):
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            r, c, aux = sw.forward(ims)
            e[1].record()
            sw.backward(ims, None, aux, g, g)
            e[2].record()
            torch.cuda.synchronize()
            tf.append(e[0].elapsed_time(e[1]))
            tb.append(e[1].elapsed_time(e[2]))
        pp = wl.pix_planes()
        fm, bm = statistics.median(tf), statistics.median(tb)
        out[name] = {"forward_ms": fm, "backward_ms": bm, "pix_planes": pp,
                     "forward_gpix_planes_s": pp / (fm * 1e-3) / 1e9,
                     "backward_gpix_planes_s": pp / (bm * 1e-3) / 1e9}
    # refinement
    wl = scenes.diff(args.seed, width=192, height=160, n_planes=64)
    imgs, rng = scenes.FrameSource(wl, device=f"cuda:{local}").frame(0, with_range=True)
    rig = Rig(ref=wl.rig.ref, cams=wl.rig.cams[1:], ref_to_cam=wl.rig.ref_to_cam[1:])
    ims = [torch.from_numpy(imgs[0].numpy().astype(np.float32) / 255.0).to(dev),
           torch.from_numpy(imgs[2].numpy().astype(np.float32) / 255.0).to(dev)]
    gt = torch.from_numpy(rng.numpy().astype(np.float32)).to(dev)
    true = rig.ref_to_cam[0]
    rs = np.random.default_rng(args.seed)
    ax, tv = rs.normal(size=3), rs.normal(size=3)
    xi0 = np.concatenate([ax / np.linalg.norm(ax) * math.radians(0.5), tv / np.linalg.norm(tv) * 0.02])
    sw = P.SoftSweep(rig, wl.levels[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    poses = refine_extrinsic(sw, ims, gt, P.se3_exp_left(xi0, true), steps=50)
    torch.cuda.synchronize()
    ref_s = time.perf_counter() - t0

    def err(p):
        dR = np.asarray(p.R) @ np.asarray(true.R).T
        return (math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(dR) - 1) / 2)))),
                float(np.linalg.norm(np.asarray(p.t) - np.asarray(true.t))))
    e0, e1 = err(poses[0]), err(poses[-1])
    main_case = out["diff-640x512-2cam-128planes"]
    line = {
        "metric": "differentiable plane sweep: forward + backward Gpix·planes/s", "unit": "Gpix·planes/s",
        "value": main_case["pix_planes"] / ((main_case["forward_ms"] + main_case["backward_ms"]) * 1e-3) / 1e9,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": main_case["forward_ms"] + main_case["backward_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "diff-640x512-2cam-128planes", "temperature": 0.05,
                   "l2": "flushed between steps (256 MB write outside the step events)"},
        "cases": out,
        "refinement": {"rig": "diff-192x160-1cam-64planes", "steps": 50, "start_deg": e0[0], "start_m": e0[1],
                       "end_deg": e1[0], "end_m": e1[1], "seconds": ref_s},
        "gpu_launches": 2 * args.steps,
    }
    print(json.dumps(line))
    return 0


def run_ringloop(args):
    """Fusion of the whole 1000-frame, 500 m ring at 2 cm voxels: the true
    range map of every frame (boxes masked) into (a) one voxel-block pool of
    2^23 blocks (32 GB) that holds the whole loop, and (b) the paper's scheme:
    a pool sized for the 60 x 3 x 60 m local map plus swap-out of the blocks
    that leave it, every 25 frames, to host memory.  Times the fusion only
    (CUDA events around each tsdf_integrate / tsdf_swap_out)."""
    import dataclasses

    import torch

    import scenes
    import paper_1809_06132_gb300 as P

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = scenes.ring(rank_seed(args.seed, rank), n_frames=1000)
    n = 1000 if args.steps >= 1000 else max(args.steps, 50)
    rend = scenes.Renderer(wl.rig.ref, ss=1, device=f"cuda:{local}")
    H, W = wl.rig.ref.height, wl.rig.ref.width
    t_r = time.time()
    depths = []
    for f in range(n):
        _, rng = rend.render(wl.scene, wl.world_to_ref[f], with_range=True)
        d = rng.to(torch.float32)
        for x0, y0, x1, y1 in wl.boxes[f]:
            d[max(0, y0):min(H, y1), max(0, x0):min(W, x1)] = 0
        depths.append(d.to(dev))
    render_s = time.time() - t_r
    out = {}
    small = dataclasses.replace(wl.tsdf, hash_slots=1 << 22, pool_blocks=1 << 20)
    for name, params, swap_every in (("whole-loop pool", wl.tsdf, 0), ("local map + swap-out", small, 25)):
        T = P.Tsdf(params, wl.rig.ref)
        host_blocks, ev_ms, peak, host_store = 0, [], 0, []
        for f in range(n):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            T.integrate(depths[f], wl.world_to_ref[f], wl.local_center(f))
            if swap_every and f % swap_every == swap_every - 1:
                k, D, Wt = T.swap_out(wl.local_center(f))        # device buffers, then to host memory
                host_store.append((k.cpu(), D.cpu(), Wt.cpu()))
                host_blocks += int(k.shape[0])
            b.record()
            ev_ms.append((a, b))
            if f % 100 == 99:
                peak = max(peak, T.count())
        torch.cuda.synchronize()
        ms = sum(x.elapsed_time(y) for x, y in ev_ms)
        st = T.status()
        out[name] = {"frames": n, "ms_per_frame": ms / n, "frames_per_s": n / (ms / 1e3), "status": st,
                     "blocks_on_gpu": T.count(), "peak_blocks_on_gpu": max(peak, T.count()),
                     "blocks_swapped_to_host": host_blocks, "pool_blocks": params.pool_blocks,
                     "gpu_voxel_bytes": params.pool_blocks * 512 * 8}
        del T
        torch.cuda.empty_cache()
    main_case = out["whole-loop pool"]
    line = {"metric": "TSDF fusion frames/s over the 1000-frame ring (2 cm voxels)", "unit": "frames/s",
            "value": main_case["frames_per_s"], "n_gpus": 1, "steps": n, "warmup": 0,
            "ms_per_step": main_case["ms_per_frame"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (true range maps of the ring, boxes masked)",
            "config": {"workload": wl.name, "voxel": 0.02, "mu": 0.1, "local_map": "60 x 3 x 60 m"},
            "cases": out, "render_s": render_s, "gpu_launches": 4 * n}
    print(json.dumps(line))
    return 0


def run_sharded(args):
    """One street sequence split over the ranks (strong scaling): each rank
    sweeps its plane range of every level of each frame, the ranks
    all-gather the per-pixel records (NCCL, plain device buffers), every
    rank merges them into the frame's depth map and fuses it into its hash
    part of the map.  Timed like the default line: CUDA events on the
    launching stream, max over ranks."""
    import torch
    import torch.distributed as dist

    import scenes
    import paper_1809_06132_gb300 as P
    from paper_1809_06132_gb300.shard import ShardedFrame

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = workload(args, args.seed)                   # the same sequence on every rank
    n_total = args.warmup + args.steps
    nf = min(n_total, 100)
    frames = render_frames(wl, nf, f"cuda:{local}")
    imgs_dev = [[torch.from_numpy(i).to(dev) for i in imgs] for imgs, _ in frames]
    H, W = wl.rig.ref.height, wl.rig.ref.width
    sw = P.Sweep(wl.rig, wl.levels, image_half=args.half)
    T = P.Tsdf(wl.tsdf, wl.rig.ref)
    depth = torch.empty((H, W), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    frame = ShardedFrame(sw, T) if world > 1 else None

    def step(i):
        f = i % nf
        if frame is not None:
            frame.step(imgs_dev[f], boxes=wl.boxes[f], world_to_ref=wl.world_to_ref[f],
                       local_center=wl.local_center(f), out=depth)
        else:
            sw.depth(imgs_dev[f], boxes=wl.boxes[f], out=depth)
            T.integrate(depth, wl.world_to_ref[f], wl.local_center(f))

    for i in range(args.warmup):
        step(i)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for k in range(args.steps):
        step(args.warmup + k)
    b.record()
    torch.cuda.synchronize()
    t1 = time.time()
    ms = max_over_ranks([a.elapsed_time(b)], dev)[0]
    clocks.stop()
    st = T.sync_status()
    line = {"metric": METRIC, "value": args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(args, wl, nf, world),
                           parallelism=f"plane ranges x{world} + record all-gather; TSDF hash parts x{world}",
                           l2="not flushed (the exchange is part of the step)"),
            "tsdf_status": st, "gpu_launches": args.steps * (2 + 1 + 2 + 4), "clocks": clocks.summary(t0, t1)}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_ringloop_swept(args):
    """A contiguous stretch of the ring (frames 0 .. n-1, 0.5 m apart) through
    the whole path: each frame's four images swept (256 full-resolution
    planes, 9x9, FP32 or FP16 image storage), boxes applied, and the swept
    depth map fused at 2 cm into the local-map pool with swap-out to host
    memory every 25 frames.  CUDA events around each frame's sweep + fusion
    (+ swap-out); the rendering of the images is outside them."""
    import dataclasses

    import torch

    import scenes
    import paper_1809_06132_gb300 as P

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = scenes.ring(rank_seed(args.seed, rank), n_frames=1000)
    n = max(10, min(args.steps, 1000))
    src = scenes.FrameSource(wl, device=f"cuda:{local}")
    sw = P.Sweep(wl.rig, wl.levels, image_half=args.half)
    params = dataclasses.replace(wl.tsdf, hash_slots=1 << 22, pool_blocks=1 << 20)
    T = P.Tsdf(params, wl.rig.ref)
    H, W = wl.rig.ref.height, wl.rig.ref.width
    depth = torch.empty((H, W), dtype=torch.float32, device=dev)
    ev, render_s, host_blocks, peak, valid = [], 0.0, 0, 0, []
    for f in range(n):
        t_r = time.time()
        imgs, _ = src.frame(f)
        im = [torch.from_numpy(np.ascontiguousarray(i.numpy())).to(dev) for i in imgs]
        torch.cuda.synchronize()
        render_s += time.time() - t_r
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record()
        sw.depth(im, boxes=wl.boxes[f], out=depth)
        b.record()
        T.integrate(depth, wl.world_to_ref[f], wl.local_center(f))
        if f % 25 == 24:
            k, D, Wt = T.swap_out(wl.local_center(f))
            host_blocks += int(k.shape[0])
            k.cpu(), D.cpu(), Wt.cpu()
        c.record()
        ev.append((a, b, c))
        if f % 10 == 9:
            valid.append(float((depth > 0).float().mean().item()))
            peak = max(peak, T.count())
    torch.cuda.synchronize()
    sweep_ms = [x.elapsed_time(y) for x, y, _ in ev]
    tsdf_ms = [y.elapsed_time(z) for _, y, z in ev]
    tot = sum(sweep_ms) + sum(tsdf_ms)
    st = T.sync_status()
    line = {"metric": "ring: swept depth + TSDF fusion frames/s (2 cm voxels, contiguous stretch of the loop)",
            "unit": "frames/s", "value": n / (tot / 1e3), "n_gpus": 1, "steps": n, "warmup": 0,
            "ms_per_step": tot / n, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (rendered ring images, swept by the library)",
            "config": {"workload": wl.name, "frames": f"0..{n - 1} of 1000 (contiguous, 0.5 m apart)",
                       "image_storage": "fp16" if args.half else "fp32", "voxel": 0.02, "mu": 0.1,
                       "local_map": "60 x 3 x 60 m, 2^20-block pool, swap-out every 25 frames"},
            "sweep_ms": {"median": statistics.median(sweep_ms), "mean": statistics.mean(sweep_ms)},
            "tsdf_ms": {"median": statistics.median(tsdf_ms), "mean": statistics.mean(tsdf_ms)},
            "blocks": {"on_gpu_end": T.count(), "peak_on_gpu": max(peak, T.count()),
                       "swapped_to_host": host_blocks},
            "depth_valid_fraction": {"mean": statistics.mean(valid) if valid else None},
            "status": st, "render_s": render_s, "gpu_launches": n * 7}
    print(json.dumps(line))
    return 0


def run_cpubase(args):
    """The FP64 oracle on the host cores for the baseline table: the tiny
    frame, and street frames 0, 50 and 99 through the whole path, each on
    every core and on one thread (one thread sweeps every 16th row of each
    level, scaled to the frame)."""
    import oracle
    import scenes
    n = os.cpu_count() or 1
    wl = scenes.street(args.seed, n_frames=100)
    out = {"cores": n}
    for f in (0, 50, 99):
        imgs, _ = scenes.FrameSource(wl, device="cuda" if _has_cuda() else "cpu").frame(f)
        imgs = [i.numpy() for i in imgs]
        t_all, _ = oracle_frame_s(wl, imgs, f, n)
        t_one, _ = oracle_frame_s(wl, imgs, f, 1, n_bands=16, bands=[7])
        out[f"street_frame_{f}"] = {f"s_{n}_threads": t_all, "s_1_thread": t_one}
    tw = scenes.tiny(args.seed)
    timgs, _ = scenes.FrameSource(tw).frame(0)
    timgs = [i.numpy() for i in timgs]
    out["tiny"] = {f"s_{n}_threads": oracle_frame_s(tw, timgs, 0, n)[0], "s_1_thread": oracle_frame_s(tw, timgs, 0, 1)[0]}
    oracle.set_threads(n)
    print(json.dumps({"metric": "FP64 oracle seconds per frame (whole path)", "data": "synthetic", **out}))
    return 0


def _has_cuda():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def main():
    args = parse()
    if args.config == "cpubase":
        return run_cpubase(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.shard:
        return run_sharded(args)
    if args.config == "batch":
        return run_batch(args)
    if args.config == "diff":
        return run_diff(args)
    if args.config == "ringloop":
        return run_ringloop_swept(args) if args.sweep_depth else run_ringloop(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
