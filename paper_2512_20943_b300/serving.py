"""Novel-view serving with continuous batching over the splatting library.

A request is one novel view (camera, resolution) of the current frame of a
streamed scene.  The anchor and the streamed frame updates stay resident on
the device: an update context decodes each frame's 16-bit update map (Sec. II
Eq. 3, Sec. III-C) every frame period and publishes the frame state into one
of two device buffers; render contexts read it with render_gaussians.

Scheduling (continuous batching): requests that have arrived wait in a queue;
whenever memory allows, the engine admits as many as fit the memory budget
(and the batch cap) into one batch and launches it as one multi-view render on
the next of several CUDA streams, so a batch's projection/ordering overlaps the
previous batch's blending on the device.  Memory frees when a batch's CUDA
event completes; the queue is re-examined continuously, so requests arriving
while others are on the GPU join the next launch.  A request larger than the
whole budget is rejected (status, not an abort).  Latency = GPU completion
time of the request's batch - arrival time, both on the engine's clock.

The plain loop renders the same request stream one view per call on one
stream, in arrival order.  Both hold Python's cyclic garbage collector off
while they serve (collections_paused), as a latency-bound server does: a full
collection over a heap of tensors and requests stalls the launching thread
for tens of milliseconds, which shows up as a p99 outlier.

Only host logic lives here; every rendering step runs in libairgs.
"""
from __future__ import annotations

import contextlib
import gc
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from .rasterizer import Rasterizer, RasterConfig


@dataclass
class Request:
    rid: int
    arrival_s: float
    viewer: int
    camera: dict
    status: str = "pending"      # pending | queued | running | done | rejected
    batch: int = -1
    done_s: float = float("nan")
    rgb: torch.Tensor | None = None

    @property
    def pixels(self) -> int:
        return int(self.camera["width"]) * int(self.camera["height"])

    @property
    def latency_ms(self) -> float:
        return 1e3 * (self.done_s - self.arrival_s)


@dataclass
class ServeStats:
    n_requests: int
    completed: int
    rejected: int
    p50_ms: float
    p99_ms: float
    mean_ms: float
    views_per_s: float
    mpix_per_s: float
    makespan_s: float
    batches: int
    mean_batch: float
    peak_bytes: int
    latencies_ms: list = field(default_factory=list)

    def to_dict(self):
        d = dict(self.__dict__)
        d.pop("latencies_ms")
        return d


def view_bytes(n_gaussians: int, camera: dict, instances_per_gaussian: float = 8.0) -> int:
    """Device memory one view holds while it is rendered: projection records
    and ordering temporaries per Gaussian, tile-list entries (estimated per
    Gaussian), the image and per-pixel state."""
    px = int(camera["width"]) * int(camera["height"])
    per_gaussian = 48 + 24          # projection record + depth key / count / sort values
    per_instance = 8 * 3            # keys, values and their ping-pong copies
    per_pixel = 12 + 4              # rgb + n_contrib
    return int(n_gaussians * (per_gaussian + instances_per_gaussian * per_instance) + px * per_pixel)


def admit_batch(queue: deque, used: int, budget: int, max_batch: int, bytes_of) -> tuple[list, int]:
    """Continuous-batching admission: take queued requests in arrival order
    while the batch cap and the memory budget allow; returns (batch, bytes)."""
    batch, bb = [], 0
    while queue and len(batch) < max_batch and used + bb + bytes_of(queue[0]) <= budget:
        r = queue.popleft()
        bb += bytes_of(r)
        batch.append(r)
    return batch, bb


def summarize(reqs, batches, peak_bytes, t_first) -> ServeStats:
    done = [r for r in reqs if r.status == "done"]
    lat = np.array([r.latency_ms for r in done]) if done else np.array([np.nan])
    end = max((r.done_s for r in done), default=t_first)
    span = max(end - t_first, 1e-9)
    return ServeStats(
        n_requests=len(reqs), completed=len(done), rejected=sum(r.status == "rejected" for r in reqs),
        p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)), mean_ms=float(lat.mean()),
        views_per_s=len(done) / span, mpix_per_s=sum(r.pixels for r in done) / span / 1e6, makespan_s=span,
        batches=batches, mean_batch=(len(done) / batches if batches else 0.0), peak_bytes=peak_bytes,
        latencies_ms=lat.tolist())


class FrameStream:
    """Device-resident ring of frame update maps, applied every `period_s`."""

    def __init__(self, maps, lo, hi, period_s: float):
        self.maps, self.lo, self.hi, self.period_s = maps, lo, hi, period_s

    def frame_at(self, t_s: float) -> int:
        return int(t_s // self.period_s)


class _Publisher:
    """Applies frame updates on its own context and publishes the frame state
    into one of two device buffers, never overwriting a buffer a running batch
    still reads."""

    def __init__(self, anchor: dict, frames: FrameStream, config: RasterConfig):
        self.stream = torch.cuda.Stream()
        self.ctx = Rasterizer(config, stream=self.stream)
        self.frames = frames
        a = anchor
        with torch.cuda.stream(self.stream):
            self.ctx.set_anchor(a["means"], a["log_scales"], a["quats"], a["opacity_logit"], a["sh"])
            self.bufs = [(a["means"].clone(), a["quats"].clone()) for _ in range(2)]
        self.shared = (a["log_scales"], a["opacity_logit"], a["sh"])
        self.current = 0
        self.frame = -1
        self.ready = torch.cuda.Event()
        self.ready.record(self.stream)
        self.readers = [[], []]  # events of batches reading each buffer

    def update_to(self, frame: int):
        if frame <= self.frame or not self.frames.maps:
            return
        nxt = 1 - self.current
        with torch.cuda.stream(self.stream):
            for ev in self.readers[nxt]:
                self.stream.wait_event(ev)
            self.readers[nxt] = []
            for f in range(self.frame + 1, frame + 1):
                m = self.frames.maps[f % len(self.frames.maps)]
                self.ctx.apply_frame_update(m, self.frames.lo, self.frames.hi, frame_id=f)
            means, quats = self.bufs[nxt]
            fm, fq = self.ctx.frame_state()
            means.copy_(fm)
            quats.copy_(fq)
            self.ready = torch.cuda.Event()
            self.ready.record(self.stream)
        self.current = nxt
        self.frame = frame

    def params(self):
        means, quats = self.bufs[self.current]
        log_scales, opacity, sh = self.shared
        return means, log_scales, quats, opacity, sh


class ServingEngine:
    """Continuous-batching novel-view server (see module docstring)."""

    def __init__(self, anchor: dict, frames: FrameStream, memory_budget_bytes: int, max_batch_views: int = 64,
                 n_streams: int = 2, config: RasterConfig | None = None, instances_per_gaussian: float = 8.0):
        self.config = config or RasterConfig()
        self.n = int(anchor["means"].shape[0])
        self.frames = frames
        self.budget = int(memory_budget_bytes)
        self.max_batch = int(max_batch_views)
        self.ipg = instances_per_gaussian
        self.pub = _Publisher(anchor, frames, self.config)
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.ctxs = [Rasterizer(self.config, stream=s) for s in self.streams]

    def bytes_of(self, req: Request) -> int:
        return view_bytes(self.n, req.camera, self.ipg)

    def _launch(self, k: int, reqs):
        s, ctx = self.streams[k], self.ctxs[k]
        cams = [r.camera for r in reqs]
        with torch.cuda.stream(s):
            s.wait_event(self.pub.ready)
            res = ctx.render_gaussians(*self.pub.params(), cams)
            done = torch.cuda.Event(enable_timing=True)
            done.record(s)
        self.pub.readers[self.pub.current].append(done)
        views = res.views()
        for r, im in zip(reqs, views):
            r.rgb = im
        return done

    def run(self, requests, keep_images: bool = False, realtime: bool = True) -> ServeStats:
        """Serve `requests` (Request list).  realtime: release each request at
        its arrival time on the engine clock; otherwise all are released at
        once and each one's arrival is the moment the engine sees it."""
        reqs = sorted(requests, key=lambda r: r.arrival_s)
        pending = deque(reqs)
        torch.cuda.synchronize()
        with collections_paused():
            return self._serve(reqs, pending, keep_images, realtime)

    def _serve(self, reqs, pending, keep_images, realtime) -> ServeStats:
        queue = deque()
        inflight = []  # (event, bytes, requests)
        used = peak = 0
        batches = 0
        rr = 0
        start = torch.cuda.Event(enable_timing=True)
        start.record()
        start.synchronize()
        t0 = time.perf_counter()
        while pending or queue or inflight:
            now = (time.perf_counter() - t0) if realtime else float("inf")
            self.pub.update_to(self.frames.frame_at(min(now, reqs[-1].arrival_s if reqs else 0.0)))
            while pending and pending[0].arrival_s <= now:
                r = pending.popleft()
                if not realtime:  # without pacing a request arrives when the engine sees it
                    r.arrival_s = time.perf_counter() - t0
                if self.bytes_of(r) > self.budget:
                    r.status = "rejected"
                else:
                    r.status = "queued"
                    queue.append(r)
            still = []
            for ev, b, rs in inflight:
                if ev.query():
                    t_done = start.elapsed_time(ev) / 1e3
                    for r in rs:
                        r.status, r.done_s = "done", t_done
                        if not keep_images:
                            r.rgb = None
                    used -= b
                else:
                    still.append((ev, b, rs))
            inflight = still
            batch, bb = admit_batch(queue, used, self.budget, self.max_batch, self.bytes_of)
            if batch:
                for r in batch:
                    r.status, r.batch = "running", batches
                used += bb
                peak = max(peak, used)
                ev = self._launch(rr % len(self.streams), batch)
                rr += 1
                batches += 1
                inflight.append((ev, bb, batch))
            elif inflight or (pending and not queue):
                time.sleep(5e-5)
        torch.cuda.synchronize()
        t_first = reqs[0].arrival_s if reqs else 0.0
        return summarize(reqs, batches, peak, t_first)


def run_plain_loop(anchor: dict, frames: FrameStream, requests, config: RasterConfig | None = None,
                   keep_images: bool = False, realtime: bool = True) -> ServeStats:
    """One view per render call, one stream, requests in arrival order."""
    config = config or RasterConfig()
    pub = _Publisher(anchor, frames, config)
    stream = torch.cuda.Stream()
    ctx = Rasterizer(config, stream=stream)
    reqs = sorted(requests, key=lambda r: r.arrival_s)
    torch.cuda.synchronize()
    with collections_paused():
        start, events = _plain_serve(reqs, pub, stream, ctx, frames, keep_images, realtime)
    torch.cuda.synchronize()
    for ev, r in events:
        r.status, r.done_s = "done", start.elapsed_time(ev) / 1e3
    t_first = reqs[0].arrival_s if reqs else 0.0
    return summarize(reqs, len(reqs), 0, t_first)


def _plain_serve(reqs, pub, stream, ctx, frames, keep_images, realtime):
    """The plain loop's launches: the start event and [(completion event, request)]."""
    start = torch.cuda.Event(enable_timing=True)
    start.record()
    start.synchronize()
    t0 = time.perf_counter()
    events = []
    for i, r in enumerate(reqs):
        if realtime:
            while time.perf_counter() - t0 < r.arrival_s:
                time.sleep(5e-5)
        now = (time.perf_counter() - t0) if realtime else r.arrival_s
        pub.update_to(frames.frame_at(now))
        if not realtime:  # without pacing a request arrives when the loop reaches it
            r.arrival_s = time.perf_counter() - t0
        with torch.cuda.stream(stream):
            stream.wait_event(pub.ready)
            res = ctx.render_gaussians(*pub.params(), [r.camera])
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
        pub.readers[pub.current].append(ev)
        r.rgb = res.views()[0] if keep_images else None
        r.status, r.batch = "running", i
        events.append((ev, r))
    return start, events


@contextlib.contextmanager
def collections_paused():
    """Automatic cyclic garbage collection off inside the block (objects are
    still freed by reference counting); the collector's previous state after."""
    was_enabled = gc.isenabled()
    gc.disable()
    try:
        yield
    finally:
        if was_enabled:
            gc.enable()


def make_requests(stream_of_tuples):
    """[(arrival_s, viewer, camera)] -> [Request]."""
    return [Request(i, float(t), int(v), cam) for i, (t, v, cam) in enumerate(stream_of_tuples)]
