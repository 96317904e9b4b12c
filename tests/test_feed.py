"""Double-buffered host feed: argument checks on the host (CPU) and, on the GPU,
that per-frame training fed from pinned host buffers through HostFeed (copies
overlapped with the previous step) gives the same losses as the same steps fed
from device buffers."""
import numpy as np
import pytest

import synthetic


def _frames(n, n_frames, w, h, n_views):
    g = synthetic.gaussians(n, 3, mean_scale=(0.7, 0.7, 0.7), log_scale=(-4.0, 0.0))
    rng = np.random.default_rng(11)
    cams = [synthetic.camera(synthetic.sphere_pose(rng, 3.0), w, h, fov_x_deg=60.0) for _ in range(n_views)]
    maps, lo, hi = [], None, None
    for t in range(n_frames):
        m, lo, hi = synthetic.update_map(n, 500 + t, size=256)
        maps.append(m)
    targets = [rng.uniform(0, 1, 3 * w * h * n_views).astype(np.float32) for _ in range(n_frames)]
    return g, cams, maps, lo, hi, targets


@pytest.mark.gpu
def test_feed_rejects_unknown_and_mismatched_buffers():
    import torch
    from paper_2512_20943_b300.feed import HostFeed
    s = torch.cuda.Stream()
    feed = HostFeed({"x": ((4,), torch.float32)}, s)
    with pytest.raises(KeyError):
        feed.put(0, y=torch.zeros(4).pin_memory())
    with pytest.raises(ValueError):
        feed.put(0, x=torch.zeros(5).pin_memory())
    with pytest.raises(KeyError):
        feed.result(0)
    with pytest.raises(KeyError):
        HostFeed({"x": ((4,), torch.float32)}, s, late=("y",))


@pytest.mark.gpu
@pytest.mark.parametrize("depth,late", [(1, False), (2, False), (3, False), (1, True), (2, True)])
def test_feed_training_matches_device_inputs(depth, late):
    """Losses of steps fed through the feed equal those of the same steps fed
    from device copies, with the targets waited for at the start of the step or
    (late) only before the backward."""
    import torch
    from paper_2512_20943_b300 import AIRGS_DELTA_PREV, Rasterizer
    from paper_2512_20943_b300.feed import HostFeed
    n, n_frames, w, h, nv = 20000, 6, 320, 240, 3
    g, cams, maps, lo, hi, targets = _frames(n, n_frames, w, h, nv)
    anchor = [torch.from_numpy(np.ascontiguousarray(g[k])).cuda()
              for k in ("means", "log_scales", "quats", "opacity_logit", "sh")]
    map_h = [torch.from_numpy(m.view(np.int16)).view(torch.uint16).pin_memory() for m in maps]
    tg_h = [torch.from_numpy(t).pin_memory() for t in targets]

    def run(fed):
        stream = torch.cuda.Stream()
        rast = Rasterizer(stream=stream)
        rast.set_anchor(*anchor)
        losses = []
        feed = HostFeed({"map": (tuple(map_h[0].shape), torch.uint16), "target": ((tg_h[0].numel(),),
                                                                              torch.float32)}, stream, depth=depth,
                        late=("target",) if late else ())
        with torch.cuda.stream(stream):
            for k in range(n_frames):
                if fed:
                    dev = feed.put(k, map=map_h[k], target=tg_h[k])
                    m_d, t_d = dev["map"], dev["target"]
                else:
                    m_d, t_d = map_h[k].cuda(), tg_h[k].cuda()
                rast.apply_frame_update(m_d, lo, hi, mode=AIRGS_DELTA_PREV, frame_id=k)
                res = rast.render(cams, save=True)
                if fed and late:
                    feed.wait(k, "target")
                loss, _ = rast.render_backward_l1(res.state, t_d)
                res.state.release()
                if fed:
                    feed.done(k, loss)
                    if k >= depth - 1:
                        losses.append(float(feed.result(k - depth + 1)[0]))
                else:
                    losses.append(float(loss))
            if fed:
                for k in range(n_frames - depth + 1, n_frames):
                    losses.append(float(feed.result(k)[0]))
        return losses

    ref = run(False)
    got = run(True)
    assert len(got) == n_frames
    # the loss is summed with atomics: equal up to the order of the additions
    np.testing.assert_allclose(got, ref, rtol=1e-5)
    assert len(set(np.round(ref, 6))) > 1  # frames differ, so a stale slot would show
