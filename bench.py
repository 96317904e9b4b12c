#!/usr/bin/env python
"""Benchmark of the AirGS splatting path on B300.

Workload (streaming training): a 300k-Gaussian SH-degree-3 anchor (means
N(0,1)*(3,2,3), log-scales N(-4,0.7), SH N(0,0.2)); each step takes frame t's
7-channel 16-bit 768x768 update map (position offset N(0,0.01), rotation
delta near identity), decodes and applies it on the device (previous-frame
mode), renders 8 views (views 8t mod 20 ... of a 20-camera 120-degree arc at
1352x1014) in one batch, and back-propagates the L1 loss against random
targets through the hand-written adjoint, accumulating the per-Gaussian blend
weight (usage frequency).  Metric: fwd+bwd Mpix/s = 8 * 1352 * 1014 / step
time.  Synthetic data (the paper's captures are not available).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs an independent
replica of the workload (the path has no data-path exchange here); the time is
the max over ranks and the value the pixels of all ranks over that time.

Inside the timed region only the two blend stages are bracketed by CUDA events
(their live times give the roofline); a second pass of a few steps with every
stage bracketed gives the breakdown.  Besides the contract's keys the line
carries: `stages` (from that pass: each stage's CUDA-event time per launch and
share, achieved GB/s of the HBM-bound stages; the blend stages also with their
timed-region times); `roofline` for the dominant kernel (algorithmic TFLOP/s
against the derived FP32 peak and the library's FFMA probe; `roofline.smem`: shared-memory TB/s against SMs x 128
B/clock and the library's LDS probe; DRAM traffic and shared-memory bytes come
from a committed ncu capture and are null once the kernel's sources change);
`e2e` (the same steps fed from pinned host buffers through the double-buffered
HostFeed, every loss read back); `serving` (served-view throughput and p50/p99
latency of the continuous-batching engine against a one-view-per-call loop,
over a 10-second request stream); `configs` (the plain 2k forward, the
per-frame 200k x 20-view step and the large 2M x 16 x 4K step with its kernel
shape autotuned, each timed the same way with its roofline fraction);
`cpu_baseline` (the FP64 oracle on this host: single-threaded, and on all
cores through its OpenMP timing build, for configs 1-3).
`--workload plain|per_frame|large` measures the other workload shapes the same
way; `--impl reference` times the oracle instead.
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
sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

METRIC = "fwd+bwd Mpix/s @300k Gaussians SH3"
UNIT = "Mpix/s"
N_GAUSS = 300_000
VIEWS_PER_STEP = 8
WIDTH, HEIGHT = 1352, 1014
MAP_SIZE = 768

# Algorithmic work per unit (see the design notes): flops per evaluated
# (pixel, Gaussian) pair of the blend forward and of the backward replay, and
# bytes per Gaussian of the projection.
# Algorithmic FP32 flops of the blending definition (exp counted apart):
# every pair of a pixel's list up to its termination is evaluated (offsets 2,
# quadratic form -(a dx^2 + c dy^2)/2 - b dx dy 9, o*G 1, clamp 1, T(1 - alpha) 2,
# with the skip and stop tests: 15 + 1 exp); a blended pair adds alpha*T and
# three colour FMAs (7) in the forward; in the replay alpha*T 1, the colour
# adjoint 5, colour gradients 6, the colour still ahead 2, dL/dalpha 3,
# dL/dpower 1, opacity 2, mean 10, conic 9, blend weight and count 2 (41).
FLOPS_TEST = 15
FLOPS_BLEND_FWD = 7
FLOPS_BLEND_BWD = 41
FLOPS_ISSUED_FWD = FLOPS_TEST + FLOPS_BLEND_FWD   # per lane evaluation the kernel issues
FLOPS_ISSUED_BWD = FLOPS_TEST + FLOPS_BLEND_BWD
FP32_LANES_PER_SM = 128

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# dominant kernels from one ncu capture of this workload (the summary and the
# command are under profiles/), keyed to the SHA-256 of the sources the kernel
# was built from: once those change the counters no longer describe it (null).
# the blend kernels, their launchers and the queue order they take items in
# (the order decides which Gaussian records are in L2 together)
_BLEND_SOURCES = ("paper_2512_20943_b300/csrc/blend_fwd.cu", "paper_2512_20943_b300/csrc/blend_bwd.cu",
                  "paper_2512_20943_b300/csrc/blend_common.cuh", "paper_2512_20943_b300/csrc/airgs_internal.cuh",
                  "paper_2512_20943_b300/csrc/kernels.h", "paper_2512_20943_b300/csrc/cull_lists.cu",
                  "paper_2512_20943_b300/csrc/api.cu")
PROFILE_STEPS = 10  # steps of the per-stage profiling pass after the timed region

NCU_TRAFFIC = {
    "blend_bwd": {"bytes_per_launch": (747.478016 + 102.799104) * 1e6, "smem_bytes_per_launch": 366248895 * 128,
                  "sources": _BLEND_SOURCES,
                  "sha256": "d8b352991546efaa8a307c7caa5531986e7045bb4df59bc3d0701b8c843eb3c1"},
    "blend_fwd": {"bytes_per_launch": (244.283904 + 228.473856) * 1e6, "smem_bytes_per_launch": 81673612 * 128,
                  "sources": _BLEND_SOURCES,
                  "sha256": "d8b352991546efaa8a307c7caa5531986e7045bb4df59bc3d0701b8c843eb3c1"},
}


# the other workload shapes' dominant kernels, from one ncu capture each (the
# commands are in profiles/per_frame_200k_sh3_20x1352x1014_ncu.md and
# profiles/plain_2k_sh0_128x128_ncu.md); the large workload is not captured
CONFIG_TRAFFIC = {
    ("per_frame", "blend_bwd"): {"bytes_per_launch": (1521.957632 + 192.448256) * 1e6, "sources": _BLEND_SOURCES,
                                 "sha256": "8dc565fa118c57211fdc94d8b39c62f02c86fc2fc92abd0e75daa87d41ae8ee2"},
    ("plain", "blend_fwd"): {"bytes_per_launch": 155.136e3, "sources": _BLEND_SOURCES,
                             "sha256": "d8b352991546efaa8a307c7caa5531986e7045bb4df59bc3d0701b8c843eb3c1"},
}


def config_traffic(kind, stage):
    rec = CONFIG_TRAFFIC.get((kind, stage))
    if not rec or _sources_sha256(rec["sources"]) != rec["sha256"]:
        return None
    return rec["bytes_per_launch"]


def _sources_sha256(paths):
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def dominant_smem_bytes(stage):
    """Shared-memory bytes per launch (ncu wavefronts x 128 B) of the same capture
    as the traffic, reported under the same source-hash rule."""
    rec = NCU_TRAFFIC.get(stage)
    if not rec or "smem_bytes_per_launch" not in rec or _sources_sha256(rec["sources"]) != rec["sha256"]:
        return None
    return rec["smem_bytes_per_launch"]


def dominant_traffic(stage):
    rec = NCU_TRAFFIC.get(stage)
    if not rec or _sources_sha256(rec["sources"]) != rec["sha256"]:
        return None
    return rec["bytes_per_launch"]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        loaded = [s for s in sm if mx and s > 0.3 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------- distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def whole_job_value(world, px_per_step, steps, max_ms):
    """Mpix/s of the whole job: the pixels every rank rendered (each rank runs
    the same per-GPU workload) over the slowest rank's time."""
    return world * px_per_step * steps / (max_ms / 1e3) / 1e6


def barrier_max(world, value, device=None):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- workload
class Workload:
    def __init__(self, n_frames, device, seed=0):
        import torch
        self.g, arc = synthetic.streaming_scene(N_GAUSS, seed)
        self.arc = arc
        # the 20 arc cameras followed by the first 8 again, so that any 8
        # consecutive views (mod 20) are one contiguous run of cameras/targets
        self.cams28 = arc + arc[:VIEWS_PER_STEP]
        tg = synthetic.target_images(arc, 1)
        tg = tg + tg[:VIEWS_PER_STEP]
        self.view_px = WIDTH * HEIGHT
        self.targets_host = np.concatenate([t.reshape(-1) for t in tg])
        self.targets = torch.from_numpy(self.targets_host).to(device)
        self.maps_host = []
        for t in range(n_frames):
            m, lo, hi = synthetic.update_map(N_GAUSS, 1000 + t, size=MAP_SIZE)
            self.maps_host.append(m)
        self.lo, self.hi = lo, hi
        self.maps = [torch.from_numpy(m.view(np.int16)).to(device).view(torch.uint16) for m in self.maps_host]
        self.params = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in self.g.items()
                       if k != "sh_degree"}

    def views(self, frame):
        s = (VIEWS_PER_STEP * frame) % len(self.arc)
        return s, self.cams28[s:s + VIEWS_PER_STEP]

    def target_slice(self, frame):
        s, _ = self.views(frame)
        n = 3 * self.view_px
        return self.targets[s * n:(s + VIEWS_PER_STEP) * n]


def train_step(rast, wl, frame, imp, map_tensor=None, target=None, before_backward=None):
    """One step of the path: decode/apply frame `frame`, batched render of its
    8 views, fused L1 backward with importance accumulation (`before_backward`
    is called between the render and the backward: the host feed's wait for
    the targets)."""
    from paper_2512_20943_b300 import AIRGS_DELTA_PREV
    m = wl.maps[frame] if map_tensor is None else map_tensor
    rast.apply_frame_update(m, wl.lo, wl.hi, mode=AIRGS_DELTA_PREV, frame_id=frame)
    _, cams = wl.views(frame)
    res = rast.render(cams, save=True)
    if before_backward is not None:
        before_backward()
    tgt = wl.target_slice(frame) if target is None else target
    loss, grads = rast.render_backward_l1(res.state, tgt, importance=imp)
    res.state.release()
    return loss, grads


# ---------------------------------------------------------------- CPU baseline (oracle)
def _crop(cam, w, h):
    """The centred w x h window of a camera (principal point moved with it)."""
    c = dict(cam)
    c["cx"] = c["cx"] - (c["width"] - w) / 2.0
    c["cy"] = c["cy"] - (c["height"] - h) / 2.0
    c["width"], c["height"] = w, h
    return c


def oracle_step(kind, impl, crop=None, frame_map=None, lo=None, hi=None, g=None, cams=None):
    """One sample of a workload on the FP64 oracle: (seconds, pixels).  kind
    "plain": the forward of config 1's scene; "train": decode/apply of one
    update map (when given) and the forward + L1 backward of the given view(s).
    impl: the oracle module (single-threaded) or its OpenMP timing build."""
    import oracle
    w = synthetic.widen(g)
    t0 = time.perf_counter()
    if frame_map is not None:
        w["means"], w["quats"] = oracle.decode_apply(frame_map, lo.astype(np.float64), hi.astype(np.float64),
                                                     w["means"], w["quats"])
    if crop is not None:
        cams = [_crop(c, min(crop, c["width"]), min(crop, c["height"])) for c in cams]
    out = impl.render(w, cams)
    if kind == "train":
        tgt = [np.random.default_rng(1).uniform(0, 1, (3, c["height"], c["width"])) for c in cams]
        _, dL = oracle.l1_loss_grad(out["rgb"], tgt)
        impl.render_backward(w, cams, dL)
    return time.perf_counter() - t0, sum(int(c["width"]) * int(c["height"]) for c in cams)


def cpu_baseline_line(crop=512):
    """The FP64 oracle timed on this host: single-threaded as it stands (the
    checker, on 512x512 crops so that it stays within seconds) and through its
    OpenMP timing build on all the host's cores (full views), for config 1 in
    full (plain 2k forward at 128x128), config 2 for one view (200k SH3, fwd + L1
    bwd) and config 3 for one frame and one view (300k SH3, decode/apply + fwd +
    L1 bwd).  value = config 3 on all cores, in the headline metric's unit."""
    import oracle
    from oracle import timing
    cores = os.cpu_count()
    usable = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else cores
    g1, c1 = synthetic.plain_forward_scene()
    g2, arc2 = synthetic.per_frame_training_scene()
    g3, arc3 = synthetic.streaming_scene(N_GAUSS, 0)
    m, lo, hi = synthetic.update_map(N_GAUSS, 1000, size=MAP_SIZE)
    samples = {
        "config1": dict(kind="plain", g=g1, cams=c1),
        "config2": dict(kind="train", g=g2, cams=arc2[:1]),
        "config3": dict(kind="train", g=g3, cams=arc3[:1], frame_map=m, lo=lo, hi=hi),
    }
    res = {"single_thread": {}, "all_cores": {}}
    for name, kw in samples.items():
        crop1 = None if name == "config1" else crop
        secs, px = oracle_step(impl=oracle, crop=crop1, **kw)
        res["single_thread"][name] = {"mpix_per_s": px / secs / 1e6, "seconds": secs, "pixels": px,
                                      "sample": "full" if crop1 is None else f"centred {crop}x{crop} crop"}
        secs, px = oracle_step(impl=timing, **kw)
        res["all_cores"][name] = {"mpix_per_s": px / secs / 1e6, "seconds": secs, "pixels": px, "sample": "full"}
    value = res["all_cores"]["config3"]["mpix_per_s"]
    return {"value": value, "unit": UNIT, "cores": cores, "usable_cores": usable, "threads": timing.threads(),
            "kind": "oracle",
            "sample": "config 3: frame 0's 768x768 uint16 map decoded/applied to the 300k SH3 anchor, then fwd + "
                      "L1 bwd of view 0 (1352x1014) on all host cores (OpenMP timing build of the oracle's source); "
                      "single_thread/all_cores give configs 1-3 (config 1 forward only)",
            **res}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    crop = 256
    g, arc = synthetic.streaming_scene(N_GAUSS, 0)
    times, pix = [], 0
    for step in range(args.warmup + args.steps):
        m, lo, hi = synthetic.update_map(N_GAUSS, 1000 + step, size=MAP_SIZE)
        view = (VIEWS_PER_STEP * step) % len(arc)
        import oracle
        secs, px = oracle_step("train", oracle, crop=crop, frame_map=m, lo=lo, hi=hi, g=g, cams=[arc[view]])
        if step >= args.warmup:
            times.append(secs)
            pix += px
    total = sum(times)
    value = pix / total / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "streaming training, 300k Gaussians SH3, 8 views 1352x1014 per step, "
                               "768x768 uint16 update maps; each reference step is one view cropped to 256x256",
                   "global_batch": 1, "seq_len": crop * crop, "parallelism": "none"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"per step: decode/apply one frame + fwd+bwd of one view cropped to {crop}x{crop}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- ours
def bits_for_tiles(n_tiles):
    return max(1, math.ceil(math.log2(max(2, n_tiles))))


def add_stage_bandwidths(stage_lines, ms, nl, n, views, n_inst, tile_bits, sh_floats=48):
    """Achieved GB/s of the HBM-bound stages from their algorithmic bytes per
    launch: decode/apply 70 B per Gaussian; projection the parameters once
    (59 + 3 + 3 + 4 + 1 floats with SH3) plus a 48 B record and 8 B of keys/counts
    per (view, Gaussian); each radix pass 4 B read (count) + 8 B read + 8 B
    written (scatter) per key (4 passes over view x Gaussian depth keys,
    ceil(tile bits / 8) over the instances); emission 8 B written per instance
    plus 52 B read per (view, Gaussian) (order, counts, record); the projection
    adjoint the parameters read and their gradients written once plus a 48 B
    record and a 48 B gradient record per (view, Gaussian)."""
    params = 4 * (3 + 3 + 4 + 1 + sh_floats)
    vn = views * n
    model = {
        "decode_apply": 70 * n,
        "project_sh": params * n + 56 * vn,
        "depth_sort": 4 * 20 * vn,
        "tile_sort": ((tile_bits + 7) // 8) * 20 * n_inst,
        "scan_emit": 8 * n_inst + 52 * vn,
        "project_bwd": 2 * params * n + 96 * vn,
    }
    for name, nbytes in model.items():
        if name in stage_lines and ms.get(name):
            per_launch = ms[name] / max(1, nl[name]) / 1e3
            launches_per_step = max(1, nl[name]) / max(1, nl.get("blend_fwd", 1))
            stage_lines[name]["gbs"] = nbytes / (per_launch * launches_per_step) / 1e9


def definition_pairs_streaming(wl, args, stream, device):
    """Definition pairs of the timed steps: (pixel, list entry) pairs of the
    full rectangle lists up to each pixel's termination (forward) and below its
    n_contrib (backward).  The timed steps list a Gaussian only in its live
    tiles, so the same frame sequence (anchor, then the warm-up and timed
    frames' updates in order) is replayed after the timed region by a context
    that builds the definition's full lists, with the pair counters on."""
    import torch
    from paper_2512_20943_b300 import RasterConfig, Rasterizer
    r = Rasterizer(RasterConfig(kernel_shape=args.shape, sort_mode=args.sort_mode, cull_lists=False), stream=stream)
    p = wl.params
    imp = (torch.zeros(N_GAUSS, dtype=torch.float32, device=device),
           torch.zeros(N_GAUSS, dtype=torch.int32, device=device))
    with torch.cuda.stream(stream):
        r.set_anchor(p["means"], p["log_scales"], p["quats"], p["opacity_logit"], p["sh"])
        for t in range(args.warmup):
            train_step(r, wl, t, imp)
        r.set_profiling(True, blend_only=True)
        r.stage_times()
        for k in range(args.steps):
            train_step(r, wl, args.warmup + k, imp)
        st = r.stage_times()
        r.set_profiling(False)
    del r
    return st["pairs_forward"], st["pairs_backward"]


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    device = torch.device("cuda", torch.cuda.current_device())
    from paper_2512_20943_b300 import RasterConfig, Rasterizer

    n_frames = args.warmup + args.steps
    wl = Workload(n_frames, device)
    stream = torch.cuda.Stream()
    rast = Rasterizer(RasterConfig(kernel_shape=args.shape, sort_mode=args.sort_mode), stream=stream)
    p = wl.params
    with torch.cuda.stream(stream):
        rast.set_anchor(p["means"], p["log_scales"], p["quats"], p["opacity_logit"], p["sh"])
        imp_w = torch.zeros(N_GAUSS, dtype=torch.float32, device=device)
        imp_c = torch.zeros(N_GAUSS, dtype=torch.int32, device=device)
    if args.autotune:
        with torch.cuda.stream(stream):
            rast.autotune(wl.views(0)[1])

    # clock sampling starts first (nvidia-smi takes a moment), then the warm-up
    # steps, so that the timed region follows busy steps instead of an idle pause
    sampler = ClockSampler(device.index)
    sampler.start()
    time.sleep(0.3)
    with torch.cuda.stream(stream):
        for t in range(args.warmup):
            train_step(rast, wl, t, (imp_w, imp_c))
    stream.synchronize()

    # timed region: per-step CUDA events on the library's stream; inside it only
    # the two blend stages carry events (the dominant kernels' live times for the
    # roofline), the per-stage breakdown comes from a second pass below
    blended0 = int(imp_c.sum(dtype=torch.int64))
    rast.set_profiling(True, blend_only=True)
    rast.stage_times()  # clear
    launches0 = Rasterizer.kernel_launch_count()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            ev[k][0].record(stream)
            train_step(rast, wl, args.warmup + k, (imp_w, imp_c))
            ev[k][1].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    launches = Rasterizer.kernel_launch_count() - launches0
    timed = rast.stage_times()
    blended = (int(imp_c.sum(dtype=torch.int64)) - blended0) / args.steps  # blended pairs per step
    # per-stage breakdown: the same frames again with every stage bracketed
    n_prof = min(args.steps, PROFILE_STEPS)
    rast.set_profiling(True)
    rast.stage_times()
    with torch.cuda.stream(stream):
        for k in range(n_prof):
            train_step(rast, wl, args.warmup + k, (imp_w, imp_c))
    stages = rast.stage_times()
    rast.set_profiling(False)
    def_fwd, def_bwd = definition_pairs_streaming(wl, args, stream, device)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    total_ms = barrier_max(world, total_ms, device)
    px_step = VIEWS_PER_STEP * WIDTH * HEIGHT
    value = whole_job_value(world, px_step, args.steps, total_ms)

    # one untimed render to read the kernel shape and list sizes the timed steps used
    with torch.cuda.stream(stream):
        res = rast.render(wl.views(args.warmup)[1], save=True)
        st = rast.stats(res.state)
        res.state.release()
    probe = {"shape": Rasterizer.shape_names()[st["kernel_shape"]], "n_instances": st["n_instances"]}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(rast, wl, args, device, stream, (imp_w, imp_c), world)

    # roofline of the dominant kernel
    peaks, peak_kind = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    n_sms = torch.cuda.get_device_properties(device).multi_processor_count
    fp32_peak = n_sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12  # TFLOP/s, FMA = 2 flops
    ms, nl = stages["ms"], stages["launches"]          # every stage, the profiling pass
    ms_t, nl_t = timed["ms"], timed["launches"]        # the blend stages, the timed region
    dom = max(ms, key=lambda k: ms[k])
    stage_lines = {}
    for name in ms:
        if nl[name] == 0:
            continue
        stage_lines[name] = {"ms_per_launch": ms[name] / nl[name], "launches_per_step": nl[name] / n_prof,
                             "share": ms[name] / max(1e-9, sum(ms.values()))}
        if nl_t[name]:
            stage_lines[name]["ms_per_launch_timed_region"] = ms_t[name] / nl_t[name]
    # Blend work (algorithmic): the definition's pairs (entries of the full
    # rectangle lists up to each pixel's termination, counted by the kernels of a
    # full-list replay of the same frames) times the test flops, plus the blended
    # pairs (the importance counts) times the blend flops.  The timed steps list a
    # Gaussian only in the tiles it can reach and the kernels decide most of the
    # remaining pairs per 8x4 block without per-pair arithmetic; the pairs of the
    # lists they walk and the lane evaluations they issue are reported beside.
    def rate(flops, name):  # over the blend stage's live event time in the timed region
        return flops / (ms_t[name] / 1e3) / 1e12 if ms_t[name] else 0.0
    def_pairs = {"forward": def_fwd, "backward": def_bwd}
    alg = {"blend_fwd": def_fwd * FLOPS_TEST + blended * args.steps * FLOPS_BLEND_FWD,
           "blend_bwd": def_bwd * FLOPS_TEST + blended * args.steps * FLOPS_BLEND_BWD}
    issued = {"blend_fwd": timed["issued_forward"] * FLOPS_ISSUED_FWD,
              "blend_bwd": timed["issued_backward"] * FLOPS_ISSUED_BWD}
    for name, key in (("blend_fwd", "forward"), ("blend_bwd", "backward")):
        if name in stage_lines:
            n_l = max(1, nl_t[name])
            stage_lines[name]["tflops_algorithmic"] = rate(alg[name], name)
            stage_lines[name]["tflops_issued_lanes"] = rate(issued[name], name)
            stage_lines[name]["definition_pairs_per_launch"] = def_pairs[key] / n_l
            stage_lines[name]["listed_pairs_per_launch"] = timed["pairs_" + key] / n_l
            stage_lines[name]["issued_evals_per_launch"] = timed["issued_" + key] / n_l
            stage_lines[name]["blended_pairs_per_launch"] = blended * args.steps / n_l
    add_stage_bandwidths(stage_lines, ms, nl, N_GAUSS, VIEWS_PER_STEP, probe["n_instances"],
                         bits_for_tiles(VIEWS_PER_STEP * math.ceil(WIDTH / 16) * math.ceil(HEIGHT / 16)))
    if dom in ("blend_bwd", "blend_fwd"):
        fl = FLOPS_BLEND_BWD if dom == "blend_bwd" else FLOPS_BLEND_FWD
        a_t = rate(alg[dom], dom)
        i_t = rate(issued[dom], dom)
        roof = {"bound": "alu", "achieved": a_t, "peak": fp32_peak, "unit": "TFLOP/s", "frac": a_t / fp32_peak,
                "traffic": dominant_traffic(dom), "kernel": "k_blend_bwd" if dom == "blend_bwd" else
                "k_blend_fwd",
                "peak_source": f"derived: {n_sms} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz ({peak_kind} max clock)",
                "work": f"{FLOPS_TEST} flops per definition pair (list entries up to termination) + {fl} per "
                        f"blended pair",
                "achieved_issued_lanes": i_t, "frac_issued_lanes": i_t / fp32_peak}
        with torch.cuda.stream(stream):
            measured = rast.measure_fp32_peak()  # an FMA probe on this GPU, after the timed region
            smem_measured = rast.measure_smem_peak()  # and a shared-memory load probe
        roof["peak_measured_fma_probe"] = measured
        roof["frac_of_measured_peak"] = a_t / measured
        # the second bound of the blend kernels: shared-memory bytes per launch from the
        # ncu capture (wavefronts x 128 B) over the live CUDA-event time of a launch
        smem_bytes = dominant_smem_bytes(dom)
        smem_peak = n_sms * 128 * sm_max * 1e6 / 1e12
        smem_tbs = smem_bytes / (ms_t[dom] / max(1, nl_t[dom]) / 1e3) / 1e12 if smem_bytes else None
        roof["smem"] = {"achieved": smem_tbs, "unit": "TB/s", "peak": smem_peak,
                        "peak_source": f"derived: {n_sms} SMs x 128 B/clock x {sm_max:.0f} MHz",
                        "frac": smem_tbs / smem_peak if smem_tbs else None,
                        "peak_measured_lds_probe": smem_measured,
                        "frac_of_measured_peak": smem_tbs / smem_measured if smem_tbs else None,
                        "bytes_per_launch": smem_bytes}
    else:
        gbs = stage_lines.get(dom, {}).get("gbs")
        roof = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": (gbs / peaks["hbm_gbs"]) if gbs else None, "traffic": None, "kernel": dom}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "streaming training: 300k-Gaussian SH3 anchor, per step one 7x768x768 uint16 "
                               "update map decoded+applied, 8 views 1352x1014 rendered in one batch, fused L1 "
                               "backward with importance accumulation",
                   "global_batch": VIEWS_PER_STEP * world, "seq_len": WIDTH * HEIGHT,
                   "parallelism": f"replicas x{world}" if world > 1 else "none",
                   "l2": "inputs larger than L2 (per step: 8.3 MB map + 131 MB targets + 236 B x 300k params "
                         "+ 115 MB projection records)"},
        "wall_s_timed": wall,
        "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": roof,
        "stages": stage_lines,
        "stages_pass": f"{n_prof} further steps of the same frames with every stage bracketed by CUDA events "
                       "(inside the timed region only the blend stages are)",
        "kernel_shape": probe["shape"],
        "instances_per_step": probe["n_instances"],
        "pairs_per_step": {"blended": blended, "forward": def_fwd / args.steps, "backward": def_bwd / args.steps,
                           "listed_forward": timed["pairs_forward"] / args.steps,
                           "listed_backward": timed["pairs_backward"] / args.steps,
                           "issued_forward": timed["issued_forward"] / args.steps,
                           "issued_backward": timed["issued_backward"] / args.steps},
    }
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_serving and world == 1:
        line["serving"] = run_serving(args, device)
    if not args.no_next_rows and world == 1:
        line["next_rows"] = run_next_rows(args, device)
    if not args.no_configs and world == 1:
        # the other workload shapes, each measured like the streaming step (plain 2k forward,
        # per-frame 200k x 20 views, large 2M x 16 x 4K with the kernel shape autotuned)
        line["configs"] = {}
        for kind, (k_steps, k_warm) in CONFIG_STEPS.items():
            c = measure_workload(kind, k_steps, k_warm, device=device)
            line["configs"][kind] = {k: c[k] for k in CONFIG_KEEP if k in c}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_line()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


WORKLOADS = {
    "plain": "plain forward render: 2,000 Gaussians SH0, one 128x128 view (forward only)",
    "per_frame": "per-frame training step: 200k Gaussians SH3, 20 views at 1352x1014 in one launch, fused L1 backward "
                 "with importance accumulation",
    "large": "large scene: 2M Gaussians SH3, 16 views at 3840x2160 in one launch, fused L1 backward with "
             "importance accumulation, kernel shape autotuned",
}


def measure_workload(kind, steps, warmup, shape=-1, sort_mode=-1, autotune=False, world=1, device=None):
    """One of the other workload shapes, timed like the streaming step: a step
    is one batched render (plain) or render + fused L1 backward with importance
    (per-frame, large) of all the workload's views; CUDA events on the
    library's stream around each step, nvidia-smi clocks sampled through the
    warm-up and the timed region, a per-stage profiling pass after it.
    Returns the bench-line fields of the workload."""
    import torch
    from paper_2512_20943_b300 import RasterConfig, Rasterizer
    if kind == "plain":
        g, cams = synthetic.plain_forward_scene()
    elif kind == "per_frame":
        g, cams = synthetic.per_frame_training_scene()
    else:
        g, cams = synthetic.large_scene()
    backward = kind != "plain"
    n = g["means"].shape[0]
    p = [torch.from_numpy(np.ascontiguousarray(g[k])).to(device)
         for k in ("means", "log_scales", "quats", "opacity_logit", "sh")]
    stream = torch.cuda.Stream()
    rast = Rasterizer(RasterConfig(kernel_shape=shape, sort_mode=sort_mode), stream=stream)
    target = None
    if backward:
        target = torch.from_numpy(np.concatenate([x.reshape(-1) for x in synthetic.target_images(cams, 1)])).to(device)
    imp = None
    if backward:  # importance counts also give the blended pairs of the roofline
        imp = (torch.zeros(n, dtype=torch.float32, device=device), torch.zeros(n, dtype=torch.int32, device=device))
    tuned = None
    with torch.cuda.stream(stream):
        if kind == "large" or autotune:
            rast.set_anchor(*p)
            shp, ms0, ms1 = rast.autotune(cams, report=True)
            tuned = {"shape": Rasterizer.shape_names()[shp], "ms_shape0": ms0, "ms_chosen": ms1,
                     "search": "coordinate search over the compiled shapes, training step timed (best of 3)"}

    def step():
        res = rast.render_gaussians(*p, cams, save=backward)
        if backward:
            rast.render_backward_l1(res.state, target, importance=imp)
            res.state.release()

    # as in the streaming step: sampling first, warm-up, a timed region whose only
    # events bracket the blend stages, then a per-stage profiling pass
    sampler = ClockSampler(device.index)
    sampler.start()
    time.sleep(0.3)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step()
    stream.synchronize()
    blended0 = int(imp[1].sum(dtype=torch.int64)) if imp is not None else 0
    rast.set_profiling(True, blend_only=True)
    rast.stage_times()
    launches0 = Rasterizer.kernel_launch_count()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for k in range(steps):
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = Rasterizer.kernel_launch_count() - launches0
    timed = rast.stage_times()
    blended = (int(imp[1].sum(dtype=torch.int64)) - blended0) / steps if imp is not None else None
    n_prof = min(steps, PROFILE_STEPS)
    rast.set_profiling(True)
    rast.stage_times()
    with torch.cuda.stream(stream):
        for _ in range(n_prof):
            step()
    stages = rast.stage_times()
    rast.set_profiling(False)
    # definition pairs (the full rectangle lists; the timed steps list only live tiles): one step of a context
    # that builds the full lists, times the steps (every step renders the same scene)
    full = Rasterizer(RasterConfig(kernel_shape=shape, sort_mode=sort_mode, cull_lists=False), stream=stream)
    full.set_profiling(True, blend_only=True)
    full.stage_times()
    with torch.cuda.stream(stream):
        res = full.render_gaussians(*p, cams, save=backward)
        if backward:
            full.render_backward_l1(res.state, target)
            res.state.release()
    fst = full.stage_times()
    del full, res
    def_pairs = {"forward": fst["pairs_forward"] * steps, "backward": fst["pairs_backward"] * steps}
    total_ms = barrier_max(world, sum(a.elapsed_time(b) for a, b in ev), device)
    px = sum(int(c["width"]) * int(c["height"]) for c in cams)
    value = whole_job_value(world, px, steps, total_ms)
    ms, nl = stages["ms"], stages["launches"]
    ms_t, nl_t = timed["ms"], timed["launches"]
    stage_lines = {name: {"ms_per_launch": ms[name] / nl[name], "launches_per_step": nl[name] / n_prof,
                          "share": ms[name] / max(1e-9, sum(ms.values()))} for name in ms if nl[name]}
    for name in stage_lines:
        if nl_t[name]:
            stage_lines[name]["ms_per_launch_timed_region"] = ms_t[name] / nl_t[name]
    with torch.cuda.stream(stream):
        res = rast.render_gaussians(*p, cams, save=True)
        st = rast.stats(res.state)
        res.state.release()
        if blended is None:  # a forward-only step: its blended pairs from one untimed render with importance
            probe = rast.render_gaussians(*p, cams, importance=True)
            blended = float(probe.importance_cnt.sum(dtype=torch.int64))
            del probe
    n_tiles = sum(math.ceil(int(c["width"]) / 16) * math.ceil(int(c["height"]) / 16) for c in cams)
    add_stage_bandwidths(stage_lines, ms, nl, n, len(cams), st["n_instances"], bits_for_tiles(n_tiles),
                         sh_floats=3 * (int(g["sh_degree"]) + 1) ** 2)
    peaks, peak_kind = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    n_sms = torch.cuda.get_device_properties(device).multi_processor_count
    fp32_peak = n_sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    line = {
        "metric": ("fwd+bwd" if backward else "fwd") + " Mpix/s", "value": value, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": total_ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[kind], "global_batch": len(cams) * world, "seq_len": px // len(cams),
                   "parallelism": f"replicas x{world}" if world > 1 else "none"},
        "gpu_launches": launches, "clocks": clocks, "stages": stage_lines,
        "stages_pass": f"{n_prof} further steps with every stage bracketed by CUDA events (inside the timed "
                       "region only the blend stages are)",
        "kernel_shape": Rasterizer.shape_names()[st["kernel_shape"]], "instances_per_step": st["n_instances"],
    }
    if tuned:
        line["autotune"] = tuned
    for name, key, fl in (("blend_fwd", "forward", FLOPS_BLEND_FWD), ("blend_bwd", "backward", FLOPS_BLEND_BWD)):
        if name in stage_lines and blended is not None and ms_t[name]:
            flops = def_pairs[key] * FLOPS_TEST + blended * steps * fl
            t_s = ms_t[name] / 1e3  # the blend stage's live event time in the timed region
            stage_lines[name]["tflops_algorithmic"] = flops / t_s / 1e12
            stage_lines[name]["frac_fp32_peak"] = flops / t_s / 1e12 / fp32_peak
        if name in stage_lines:
            stage_lines[name]["definition_pairs_per_launch"] = def_pairs[key] / max(1, nl_t[name])
            stage_lines[name]["listed_pairs_per_launch"] = timed["pairs_" + key] / max(1, nl_t[name])
            stage_lines[name]["issued_evals_per_launch"] = timed["issued_" + key] / max(1, nl_t[name])
    dom = max(stage_lines, key=lambda k: stage_lines[k]["share"])
    if dom in ("blend_bwd", "blend_fwd") and "tflops_algorithmic" in stage_lines[dom]:
        bl = stage_lines[dom]
        traffic = config_traffic(kind, dom)
        line["roofline"] = {"bound": "alu", "achieved": bl["tflops_algorithmic"], "peak": fp32_peak,
                            "unit": "TFLOP/s", "frac": bl["frac_fp32_peak"], "traffic": traffic,
                            "kernel": "k_blend_bwd" if dom == "blend_bwd" else "k_blend_fwd",
                            "peak_source": f"derived: {n_sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                           f"{sm_max:g} MHz"}
        if traffic is None:
            line["roofline"]["traffic_note"] = "no ncu capture of this workload with the current kernel sources"
    else:
        gbs = stage_lines[dom].get("gbs")
        line["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                            "frac": (gbs / peaks["hbm_gbs"]) if gbs else None, "traffic": None, "kernel": dom}
    line["dominant_stage"] = dom
    del rast, p, target, imp
    torch.cuda.empty_cache()
    return line


def run_config(args):
    """The other workload shapes with the same timing, stage profiling and
    roofline (one GPU; replicas under torchrun like the streaming step)."""
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    device = torch.device("cuda", torch.cuda.current_device())
    line = measure_workload(args.workload, args.steps, args.warmup, args.shape, args.sort_mode, args.autotune, world,
                            device)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# steps of the other workload shapes inside the default run (their timed work stays a few seconds)
CONFIG_STEPS = {"plain": (20, 5), "per_frame": (10, 3), "large": (3, 3)}
CONFIG_KEEP = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "clocks", "roofline", "dominant_stage",
               "kernel_shape", "autotune", "config", "gpu_launches")


def run_serving(args, device):
    """Served-view latency of the continuous-batching engine vs the plain
    one-view-per-launch loop on the serving workload: 500k-Gaussian SH3 anchor
    with 30 fps frame updates resident on the device, 64 viewers issuing
    Poisson requests (30/s each) at 640x480 / 1280x720 / 1920x1080 from poses on
    a 3 m sphere, admission by a memory budget that binds at peak."""
    import torch
    from paper_2512_20943_b300.serving import FrameStream, ServingEngine, make_requests, run_plain_loop, view_bytes
    n = 500_000
    g = synthetic.serving_scene(n)
    anchor = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in g.items() if k != "sh_degree"}
    maps = []
    for t in range(30):
        m, lo, hi = synthetic.update_map(n, 2000 + t, size=MAP_SIZE)
        maps.append(torch.from_numpy(m.view(np.int16)).to(device).view(torch.uint16))
    frames = FrameStream(maps, lo, hi, period_s=1.0 / 30.0)
    stream = synthetic.serving_requests(n_viewers=64, rate_hz=30.0, duration_s=args.serve_seconds, seed=4)
    budget = 24 * view_bytes(n, dict(width=1920, height=1080))
    # warm-up of the engine that then serves (as a server warms up before it
    # takes traffic): a few batches so that its memory pools and kernels are ready
    eng = ServingEngine(anchor, frames, budget, max_batch_views=64)
    warm = make_requests([(0.0, 0, c) for _, _, c in stream[:16]])
    eng.run(warm, realtime=False)
    st_eng = eng.run(make_requests(stream), realtime=True)
    st_plain = run_plain_loop(anchor, frames, make_requests(stream), realtime=True)
    keep = ("n_requests", "completed", "rejected", "p50_ms", "p99_ms", "mean_ms", "views_per_s", "mpix_per_s",
            "batches", "mean_batch", "peak_bytes", "makespan_s")
    return {
        "workload": f"500k Gaussians SH3, 64 viewers x Poisson 30/s for {args.serve_seconds:g} s, sizes 640x480/"
                    "1280x720/1920x1080, 30 fps frame updates on device, memory budget "
                    f"{budget / 2**30:.2f} GiB",
        "continuous_batching": {k: getattr(st_eng, k) for k in keep},
        "plain_loop": {k: getattr(st_plain, k) for k in keep},
    }


NEXT_REPS = 20  # timed calls per kernel of the next_rows block (each after an L2 flush and a device spin)
SSIM_FLOPS_PER_VALUE = 5 * 44 + 3 * 44 + 40 + 6  # the D-SSIM loss and gradient, separable form


SLEEP_CYCLES = 300_000  # about 0.15 ms of device spin before each timed call


def _timed_calls(stream, fn, reps, flush):
    """Mean device time (ms) of fn() on the library's stream: reps calls, each
    after writing a buffer larger than L2 and a short device spin (both outside
    the events), so that the call's kernels are all queued by the time the
    stream reaches the first event and its host work (argument checks,
    allocations) does not count as device time."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(3):
            fn()
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    with torch.cuda.stream(stream):
        for a, b in ev:
            flush.zero_()
            torch.cuda._sleep(SLEEP_CYCLES)
            a.record(stream)
            fn()
            b.record(stream)
    stream.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in ev)


def run_next_rows(args, device):
    """The widened rows on the streaming workload's data (300k Gaussians SH3,
    frame 0's update applied, the 8 views of step 0 at 1352x1014): usage-
    frequency pruning of the frame delta (Sec. III-C), the pruning-level space
    and Algorithm 1's choice, the densification statistics and the clone /
    split / discard step of keyframe reconstruction (Sec. III-B) and the D-SSIM
    term of L_3DGS (Eq. 1).  Device times from CUDA events, each call after an
    L2 flush and a device spin (_timed_calls); HBM-bound kernels as algorithmic
    bytes over that time against the measured copy bandwidth."""
    import torch
    from paper_2512_20943_b300 import AIRGS_DELTA_ANCHOR, RasterConfig, Rasterizer
    from paper_2512_20943_b300.pruning import pruning_level_space, select_pruning_level
    peaks, _ = measured_peaks()
    hbm = peaks["hbm_gbs"]
    n = N_GAUSS
    g, arc = synthetic.streaming_scene(n, 0)
    cams = arc[:VIEWS_PER_STEP]
    stream = torch.cuda.Stream()
    rast = Rasterizer(RasterConfig(), stream=stream)
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in g.items() if k != "sh_degree"}
    p = (t["means"], t["log_scales"], t["quats"], t["opacity_logit"], t["sh"])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    n_px = VIEWS_PER_STEP * WIDTH * HEIGHT
    target = torch.from_numpy(np.concatenate([x.reshape(-1) for x in synthetic.target_images(cams, 1)])).to(device)
    out = {"workload": f"{n // 1000}k Gaussians SH3, {VIEWS_PER_STEP} views {WIDTH}x{HEIGHT} (the streaming step's)",
           "timing": f"CUDA events around each call on the library's stream, mean of {NEXT_REPS}, a 256 MB write "
                     "(inputs out of L2) and a 0.15 ms device spin (the call's host work queued behind it) "
                     "before each", "hbm_peak_gbs": hbm}

    def rate(bytes_, ms):
        gbs = bytes_ / (ms * 1e-3) / 1e9
        return {"ms": ms, "bytes": bytes_, "gbs": gbs, "frac_hbm": gbs / hbm}

    with torch.cuda.stream(stream):
        rast.set_anchor(*p)
        w, _ = rast.gaussian_importance(cams)
    stream.synchronize()
    rng = np.random.default_rng(7)
    D = torch.from_numpy(rng.normal(0, 0.01, (7, n)).astype(np.float32)).to(device)
    D_sent = torch.zeros(7, n, dtype=torch.float32, device=device)

    # f1: usage-frequency pruning p(D_t - D'_{t-1}) of 30 % of the Gaussians
    n_prune = int(0.3 * n)
    keep = rast.prune_mask(w, n_prune)
    ms_mask = _timed_calls(stream, lambda: rast.prune_mask(w, n_prune), NEXT_REPS, flush)
    ms_delta = _timed_calls(stream, lambda: rast.prune_delta(D, D_sent.clone(), keep), NEXT_REPS, flush)
    ms_clone = _timed_calls(stream, lambda: D_sent.clone(), NEXT_REPS, flush)
    d, _ = rast.prune_delta(D, D_sent.clone(), keep)
    ms_apply = _timed_calls(stream, lambda: rast.apply_frame_delta(d, mode=AIRGS_DELTA_ANCHOR, quat_add=True),
                            NEXT_REPS, flush)
    out["pruning"] = {
        "fraction": 0.3,
        # mask: the weights read, the mask written (the sort inside is the implementation's)
        "prune_mask": rate(n * (4 + 1), ms_mask),
        # delta: D_t, the transmitted record and the mask read; the delta and the record written
        "prune_delta": rate(n * (28 + 28 + 1 + 28 + 28), max(ms_delta - ms_clone, 1e-6)),
        # apply: the delta and the anchor's means and quaternions read, the frame's written
        "apply_frame_delta": rate(n * (28 + 28 + 28), ms_apply),
    }

    # f3: densification statistics (sum over views of |dL/d mean2d| and the view count) in the
    # projection adjoint, and the selection
    dg = torch.zeros(n, dtype=torch.float32, device=device)
    dv = torch.zeros(n, dtype=torch.int32, device=device)

    def bwd(dens):
        res = rast.render_gaussians(*p, cams, save=True)
        rast.render_backward_ex(res.state, target=target, densify=(dg, dv) if dens else None)
        res.state.release()

    ms_with = _timed_calls(stream, lambda: bwd(True), NEXT_REPS, flush)
    ms_without = _timed_calls(stream, lambda: bwd(False), NEXT_REPS, flush)
    ms_sel = _timed_calls(stream, lambda: rast.densify_select(dg, dv, 1e-4), NEXT_REPS, flush)
    # the clone / split / discard step: the 10 % of the visible Gaussians with the largest mean
    # screen-space gradient selected, size threshold at the median largest scale (about half the
    # selected Gaussians split), opacity floor 0.005, standard normal samples
    with torch.cuda.stream(stream):
        vis = dv > 0
        thr_g = float(torch.quantile((dg[vis] / dv[vis].float()).double(), 0.9)) if bool(vis.any()) else 1e-4
        sel = rast.densify_select(dg, dv, thr_g)
        size_thr = float(torch.exp(p[1].max(dim=1).values.median()).item())
        z = torch.randn(n, 2, 3, generator=torch.Generator(device=device).manual_seed(31), device=device)
        dens = rast.densify_apply(*p, sel, z, size_thr, 1.6, 0.005)
    m_out, n_sel = int(dens["parent"].numel()), int(sel.sum().item())
    # the split Gaussians (selected, alive, some log scale above the threshold; float32 compares)
    lo_thr = float(np.log(0.005 / (1.0 - 0.005)))
    n_split = int((sel.bool() & (p[1] > float(np.log(size_thr))).any(dim=1) & ~(p[3] < lo_thr)).sum().item())
    del dens
    ms_apply_dens = _timed_calls(stream, lambda: rast.densify_apply(*p, sel, z, size_thr, 1.6, 0.005, read_count=False),
                                 NEXT_REPS, flush)
    K3 = 3 * p[4].shape[1]
    out["densification"] = {
        "render_and_backward_ms_with_statistics": ms_with,
        "render_and_backward_ms_without": ms_without,
        "densify_select": rate(n * (4 + 4 + 1), ms_sel),
        # apply: every input Gaussian and its selection byte read once, the split ones' samples,
        # every output Gaussian and its parent index written
        "densify_apply": dict(rate(n * (44 + 4 * K3 + 1) + n_split * 24 + m_out * (44 + 4 * K3 + 4), ms_apply_dens),
                              n_in=n, selected=n_sel, split=n_split, n_out=m_out, size_threshold=size_thr,
                              min_opacity=0.005),
    }

    # f2: the pruning-level space S_t^d (11 levels: mask, delta, apply, render of the 8 views and
    # its squared error against the unpruned render, per level) and Algorithm 1's choice at a
    # budget of half the unpruned delta per frame (host wall time: the level loop reads each
    # level's error and size back)
    with torch.cuda.stream(stream):
        pruning_level_space(rast, D, D_sent, w, cams)  # warm
    stream.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        space = pruning_level_space(rast, D, D_sent, w, cams)
    stream.synchronize()
    ms_space = (time.perf_counter() - t0) * 1e3
    levels = [(min(lv.quality, 200.0), lv.size) for lv in space]
    t0 = time.perf_counter()
    chosen = select_pruning_level(levels, 2.0, 0.5 * space[0].size, 1.0)
    ms_select = (time.perf_counter() - t0) * 1e3
    out["level_selection"] = {
        "levels": len(space), "space_ms_wall": ms_space, "select_ms_host": ms_select, "chosen": chosen,
        "budget": "B/R = half the unpruned delta's bytes", "psnr_db": [round(q, 2) for q, _ in levels],
        "bytes": [sz for _, sz in levels],
    }

    # f4: L_3DGS = 0.8 L1 + 0.2 (1 - SSIM) and its image gradient over the 8 rendered views, and a
    # training step with it (render, loss, explicit-gradient backward) beside the fused-L1 step
    res = rast.render_gaussians(*p, cams)
    rgb = res.rgb
    ms_loss = _timed_calls(stream, lambda: rast.l3dgs_loss(cams, rgb, target, 0.2), NEXT_REPS, flush)
    imp = (torch.zeros(n, dtype=torch.float32, device=device), torch.zeros(n, dtype=torch.int32, device=device))

    def step_l3dgs():
        r = rast.render_gaussians(*p, cams, save=True)
        _, grad = rast.l3dgs_loss(cams, r.rgb, target, 0.2)
        rast.render_backward(r.state, grad, importance=imp)
        r.state.release()

    def step_l1():
        r = rast.render_gaussians(*p, cams, save=True)
        rast.render_backward_l1(r.state, target, importance=imp)
        r.state.release()

    ms_step_ssim = _timed_calls(stream, step_l3dgs, NEXT_REPS, flush)
    ms_step_l1 = _timed_calls(stream, step_l1, NEXT_REPS, flush)
    # issue-bound: per value (pixel and channel) the separable 11-tap correlations of the five
    # moments and of the three partials, each a horizontal and a vertical pass (11 FMAs each),
    # the SSIM map and its partials, and the combination: 5 x 44 + 3 x 44 + 40 + 6 flops
    n_sms = torch.cuda.get_device_properties(device).multi_processor_count
    fp32_peak = n_sms * FP32_LANES_PER_SM * 2 * float(peaks.get("sm_max_mhz", 2032.0)) * 1e6 / 1e12
    flops = n_px * 3 * SSIM_FLOPS_PER_VALUE
    loss_rate = {"ms": ms_loss, "mpix_per_s": n_px / (ms_loss * 1e-3) / 1e6, "bound": "alu",
                 "tflops_algorithmic": flops / (ms_loss * 1e-3) / 1e12,
                 "frac_fp32": flops / (ms_loss * 1e-3) / 1e12 / fp32_peak, "fp32_peak_tflops": fp32_peak,
                 "hbm_bytes": n_px * 3 * (4 + 4 + 4)}  # image and target read, gradient written
    out["d_ssim"] = {
        "lambda": 0.2, "loss_and_gradient": loss_rate,
        "training_step_ms_l3dgs": ms_step_ssim, "training_step_ms_fused_l1": ms_step_l1,
        "training_mpix_per_s_l3dgs": n_px / (ms_step_ssim * 1e-3) / 1e6,
    }
    del rast, flush
    torch.cuda.empty_cache()
    return out


def run_e2e(rast, wl, args, device, stream, imp, world):
    """Same step through the public API with host inputs: every step the frame's
    update map and its 8 target images are copied from pinned host memory, and
    its loss is copied back and read on the host.  The copies go through the
    package's double-buffered HostFeed, so step k's inputs cross PCIe while step
    k - 1 computes, the targets (read only by the backward) are waited for after
    the render, and step k - 1's loss is read while step k runs; the timed region
    ends when the last step's loss has been read."""
    import torch
    from paper_2512_20943_b300.feed import HostFeed
    map_h = [torch.from_numpy(m.view(np.int16)).view(torch.uint16).pin_memory() for m in wl.maps_host]
    n = 3 * wl.view_px * VIEWS_PER_STEP
    tg_h = torch.from_numpy(wl.targets_host).pin_memory()
    feed = HostFeed({"map": (tuple(map_h[0].shape), torch.uint16), "target": ((n,), torch.float32)}, stream,
                    device=device, late=("target",))
    losses = []

    def step(k, frame):
        s, _ = wl.views(frame)
        dev = feed.put(k, map=map_h[frame], target=tg_h[s * 3 * wl.view_px:s * 3 * wl.view_px + n])
        loss, _ = train_step(rast, wl, frame, imp, map_tensor=dev["map"], target=dev["target"],
                             before_backward=lambda: feed.wait(k, "target"))
        feed.done(k, loss)
        if k:
            losses.append(float(feed.result(k - 1)[0]))

    with torch.cuda.stream(stream):
        n_warm = min(args.warmup, len(map_h))
        for k in range(n_warm):
            step(k, k)
        if n_warm:
            losses.append(float(feed.result(n_warm - 1)[0]))
        torch.cuda.synchronize()
        losses.clear()
        t0 = time.perf_counter()
        for k in range(args.steps):
            step(k, (args.warmup + k) % len(map_h))
        losses.append(float(feed.result(args.steps - 1)[0]))
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
    assert len(losses) == args.steps and all(np.isfinite(losses))
    secs = barrier_max(world, secs, device)
    value = world * VIEWS_PER_STEP * WIDTH * HEIGHT * args.steps / secs / 1e6
    return {"value": value, "unit": UNIT, "h2d_bytes_per_step": feed.h2d_bytes, "d2h_bytes_per_step": 4,
            "ms_per_step": 1e3 * secs / args.steps, "overlap": "double-buffered: inputs of step k copied while "
                                                              "step k - 1 computes, targets awaited before the "
                                                              "backward; every loss read back"}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="length of the served request stream")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workload shapes in the default line")
    ap.add_argument("--no-next-rows", action="store_true",
                    help="skip the pruning / level-selection / densification / D-SSIM timings")
    ap.add_argument("--autotune", action="store_true", help="search the kernel shapes first and keep the fastest")
    ap.add_argument("--shape", type=int, default=-1, help="kernel shape (-1: autotuned choice or shape 0)")
    ap.add_argument("--sort-mode", type=int, default=-1,
                    help="0: global radix ordering; 1: per-tile ordering when lists fit; -1: per-tile for small batches")
    ap.add_argument("--workload", choices=["streaming"] + sorted(WORKLOADS), default="streaming",
                    help="streaming (the default line) or another workload shape, reported the same way")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "streaming":
        return run_config(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
