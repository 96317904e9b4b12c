"""Parity at full workload sizes, in the launch configuration the benchmark
uses: the GPU renders (and back-propagates) every view of a batch in one
launch; the oracle computes sampled windows of full views (same cameras, every
Gaussian projected and binned, only the window's pixels blended / replayed).
Bars as in test_gpu_parity: RGB 1e-3 absolute on unflagged pixels, gradients
1e-3 relative with the loss restricted to the windows."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests._helpers import RGB_ATOL, assert_grad_close, params, to_cuda, views_np

pytestmark = pytest.mark.gpu


def window_loss(cams, windows, ref, seed):
    """Random dL/d(rgb) inside the windows (zero outside and on flagged pixels)."""
    rng = np.random.default_rng(seed)
    out = []
    for v, c in enumerate(cams):
        d = np.zeros((3, c["height"], c["width"]))
        x0, y0, x1, y1 = windows[v]
        if x1 > x0:
            d[:, y0:y1, x0:x1] = rng.standard_normal((3, y1 - y0, x1 - x0))
            d[:, ref["ambig"][v]] = 0.0
        out.append(d)
    return out


def check_windows(rgb_views, ref, windows):
    for v, (x0, y0, x1, y1) in enumerate(windows):
        if x1 <= x0:
            continue
        ok = ~ref["ambig"][v][y0:y1, x0:x1]
        assert ok.mean() > 0.95, v
        err = np.abs(rgb_views[v][:, y0:y1, x0:x1] - ref["rgb"][v][:, y0:y1, x0:x1])[:, ok].max()
        assert err < RGB_ATOL, (v, err)


def run_case(rast, g_frame, cams, windows, seed, grads=True):
    """GPU forward (+ explicit-dL backward) of all views in one launch vs the
    oracle on the windowed views only (the GPU's loss is zero elsewhere)."""
    t = to_cuda(g_frame)
    res = rast.render_gaussians(*params(t), cams, T=True, save=True)
    torch.cuda.synchronize()
    gw = synthetic.widen(g_frame)
    sel = [v for v, w in enumerate(windows) if w[2] > w[0]]
    sub_cams, sub_win = [cams[v] for v in sel], [windows[v] for v in sel]
    ref = oracle.render(gw, sub_cams, windows=sub_win)
    rgb = views_np(res.rgb, cams)
    check_windows([rgb[v] for v in sel], ref, sub_win)
    Tv = views_np(res.T, cams, 1)
    for v in range(len(cams)):
        assert (rgb[v] >= 0).all() and (Tv[v] >= 0).all() and (Tv[v] <= 1).all()
    if grads:
        dL_sub = window_loss(sub_cams, sub_win, ref, seed)
        dL = [np.zeros((3, c["height"], c["width"])) for c in cams]
        for k, v in enumerate(sel):
            dL[v] = dL_sub[k]
        flat = torch.from_numpy(np.concatenate([d.reshape(-1) for d in dL]).astype(np.float32)).cuda()
        gr = rast.render_backward(res.state, flat)
        torch.cuda.synchronize()
        ref_g = oracle.render_backward(gw, sub_cams, dL_sub, windows=sub_win)
        for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
            assert_grad_close(gr[k].cpu().numpy(), ref_g[k], k)
    res.state.release()
    return res


def no_window():
    return (0, 0, 0, 0)


def test_streaming_training_batch_full_size():
    """300k-Gaussian SH3 anchor, frame 0's 768x768 uint16 update decoded on the
    device, 8 views at 1352x1014 in one batch (the benchmark step)."""
    from paper_2512_20943_b300 import Rasterizer
    g, arc = synthetic.streaming_scene()
    t = to_cuda(g)
    rast = Rasterizer()
    rast.set_anchor(*params(t))
    m, lo, hi = synthetic.update_map(300_000, 1000, size=768)
    rast.apply_frame_update(torch.from_numpy(m.view(np.int16)).cuda().view(torch.uint16), lo, hi)
    means, quats = (x.cpu().numpy() for x in rast.frame_state())
    frame = dict(g, means=means, quats=quats)
    cams = arc[0:8]
    windows = [no_window()] * 8
    windows[0] = (620, 460, 700, 540)   # dense centre
    windows[5] = (40, 40, 104, 104)     # sparse corner
    windows[7] = (1300, 990, 1352, 1014)  # ragged bottom-right edge
    run_case(rast, frame, cams, windows, seed=1)


def test_per_frame_training_20_views_full_size():
    """200k Gaussians SH3, 20 views at 1352x1014 in one launch."""
    from paper_2512_20943_b300 import Rasterizer
    g, cams = synthetic.per_frame_training_scene()
    windows = [no_window()] * 20
    windows[0] = (500, 400, 564, 464)
    windows[19] = (900, 300, 964, 364)
    run_case(Rasterizer(), g, cams, windows, seed=2)


def test_large_scene_16_views_4k_full_size():
    """2M Gaussians SH3, 16 views at 3840x2160 in one launch with importance,
    after autotuning the blend variant; forward windows and gradients on one."""
    from paper_2512_20943_b300 import Rasterizer
    g, cams = synthetic.large_scene()
    rast = Rasterizer()
    t = to_cuda(g)
    rast.set_anchor(*params(t))
    variant = rast.autotune(cams)
    assert 0 <= variant < len(Rasterizer.variant_names())
    windows = [no_window()] * 16
    windows[8] = (1880, 1040, 1944, 1104)
    run_case(rast, g, cams, windows, seed=3)
    # usage frequency over all 16 views: forward and backward replay agree
    res = rast.render_gaussians(*params(t), cams, importance=True, save=True)
    iw = torch.zeros_like(res.importance_w)
    ic = torch.zeros_like(res.importance_cnt)
    rast.render_backward(res.state, torch.zeros_like(res.rgb), importance=(iw, ic))
    torch.cuda.synchronize()
    assert torch.equal(ic, res.importance_cnt)
    assert int(ic.sum()) > 0
    res.state.release()
