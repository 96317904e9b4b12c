"""Serving loop: admission logic on the host (CPU) and, on the GPU, that a view
rendered alone equals the same view rendered in a mixed batch, and that the
continuous-batching engine and the plain loop serve a request stream."""
from collections import deque

import numpy as np
import pytest

import synthetic


def test_admit_batch_respects_budget_order_and_cap():
    from paper_2512_20943_b300.serving import admit_batch
    q = deque([("a", 5), ("b", 3), ("c", 4), ("d", 1)])
    size = lambda r: r[1]
    batch, b = admit_batch(q, used=0, budget=9, max_batch=10, bytes_of=size)
    assert [r[0] for r in batch] == ["a", "b"] and b == 8  # c would exceed; order kept (no skipping)
    assert [r[0] for r in q] == ["c", "d"]
    batch, b = admit_batch(q, used=8, budget=9, max_batch=10, bytes_of=size)
    assert batch == [] and b == 0  # nothing fits until memory frees
    batch, b = admit_batch(q, used=0, budget=100, max_batch=1, bytes_of=size)
    assert [r[0] for r in batch] == ["c"]


def test_view_bytes_grows_with_resolution_and_gaussians():
    from paper_2512_20943_b300.serving import view_bytes
    small = view_bytes(1000, dict(width=640, height=480))
    big = view_bytes(1000, dict(width=1920, height=1080))
    assert big - small == (1920 * 1080 - 640 * 480) * 16
    assert view_bytes(2000, dict(width=640, height=480)) > small


def test_summary_percentiles():
    from paper_2512_20943_b300.serving import Request, summarize
    reqs = [Request(i, 0.0, 0, dict(width=10, height=10)) for i in range(100)]
    for i, r in enumerate(reqs):
        r.status, r.done_s = "done", (i + 1) / 1000.0
    s = summarize(reqs, batches=10, peak_bytes=0, t_first=0.0)
    assert s.completed == 100 and abs(s.p50_ms - 50.5) < 1e-9 and abs(s.p99_ms - 99.01) < 1e-6
    assert abs(s.views_per_s - 1000.0) < 1e-6 and s.mean_batch == 10


def test_collections_paused_restores_the_collector():
    import gc
    from paper_2512_20943_b300.serving import collections_paused
    was = gc.isenabled()
    try:
        gc.enable()
        with collections_paused():
            assert not gc.isenabled()
        assert gc.isenabled()
        with pytest.raises(RuntimeError):  # restored on an exception too
            with collections_paused():
                raise RuntimeError("stop")
        assert gc.isenabled()
        gc.disable()  # a caller that had it off keeps it off
        with collections_paused():
            assert not gc.isenabled()
        assert not gc.isenabled()
    finally:
        (gc.enable if was else gc.disable)()


def _scene(n=20000):
    import torch
    g = synthetic.gaussians(n, 3, mean_scale=(0.7, 0.7, 0.7), log_scale=(-4.0, 0.6))
    anchor = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in g.items() if k != "sh_degree"}
    maps = []
    for t in range(3):
        m, lo, hi = synthetic.update_map(n, 1000 + t, size=256)
        maps.append(torch.from_numpy(m.view(np.int16)).cuda().view(torch.uint16))
    return anchor, maps, lo, hi


@pytest.mark.gpu
def test_view_alone_equals_view_in_mixed_batch():
    import torch
    from paper_2512_20943_b300 import Rasterizer
    anchor, _, _, _ = _scene()
    rng = np.random.default_rng(5)
    cams = [synthetic.camera(synthetic.sphere_pose(rng, 3.0), w, h, fov_x_deg=60.0)
            for (w, h) in [(640, 480), (1280, 720), (320, 200), (1920, 1080)]]
    rast = Rasterizer()
    p = (anchor["means"], anchor["log_scales"], anchor["quats"], anchor["opacity_logit"], anchor["sh"])
    mixed = rast.render_gaussians(*p, cams).views()
    for k, cam in enumerate(cams):
        alone = rast.render_gaussians(*p, [cam]).views()[0]
        assert torch.equal(alone, mixed[k]), k  # no atomics in the forward image: bit-identical
    assert float(mixed[3].max()) > 0.05


@pytest.mark.gpu
def test_engine_serves_stream_and_matches_plain_loop():
    import torch
    from paper_2512_20943_b300.serving import FrameStream, ServingEngine, make_requests, run_plain_loop, view_bytes
    anchor, maps, lo, hi = _scene()
    frames = FrameStream(maps, lo, hi, period_s=1.0 / 30.0)
    rng = np.random.default_rng(9)
    stream = []
    for i in range(60):
        w, h = [(160, 120), (320, 180), (480, 270)][i % 3]
        stream.append((i * 0.004, i % 8, synthetic.camera(synthetic.sphere_pose(rng, 3.0), w, h, fov_x_deg=60.0)))
    huge = synthetic.camera((0, 0, -3.0), 16384, 16384, fov_x_deg=60.0)
    stream.append((0.1, 0, huge))  # larger than the whole budget: rejected
    budget = 4 * view_bytes(20000, dict(width=480, height=270))
    eng = ServingEngine(anchor, frames, memory_budget_bytes=budget, max_batch_views=8)
    reqs = make_requests(stream)
    st = eng.run(reqs, keep_images=True, realtime=False)
    assert st.completed == 60 and st.rejected == 1
    assert st.batches < 60 and st.peak_bytes <= budget
    assert np.isfinite(st.p50_ms) and st.p99_ms >= st.p50_ms > 0
    # without real-time pacing every request sees the frame state of the last
    # arrival; the plain loop renders the same views one per call
    plain_reqs = make_requests(stream[:-1])
    frames2 = FrameStream(maps, lo, hi, period_s=1e9)  # frame 0 only: compare images exactly
    eng2 = ServingEngine(anchor, frames2, memory_budget_bytes=budget, max_batch_views=8)
    r2 = make_requests(stream[:-1])
    eng2.run(r2, keep_images=True, realtime=False)
    run_plain_loop(anchor, frames2, plain_reqs, keep_images=True, realtime=False)
    for a, b in zip(r2, plain_reqs):
        assert torch.equal(a.rgb, b.rgb), a.rid
    # an engine serves again after a run (the benchmark warms the engine it
    # measures): same images the second time
    r3 = make_requests(stream[:-1])
    eng2.run(r3, keep_images=True, realtime=False)
    for a, b in zip(r2, r3):
        assert torch.equal(a.rgb, b.rgb), a.rid
