"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: tile lists bit-exact (when the oracle bins the GPU's own single-precision
centres, radii and depths), RGB within 1e-3 absolute, gradients within 1e-3
relative (per tensor L2, plus 1e-3 of the largest magnitude elementwise),
importance counts exact; pixels whose blend passes within the oracle's
tolerance of a threshold (alpha_min, T_min, power = 0, near-equal depths) are
excluded from exact comparisons and must be rare.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests._helpers import (RGB_ATOL, assert_grad_close, params, small_sh3_scene, to_cuda, views_np)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rast():
    """The radix ordering the benchmark's batch sizes take (the default picks
    the per-tile ordering for batches this small; both are tested), with the
    definition's full rectangle lists (saved states of a culling context hold
    only the live tiles)."""
    from paper_2512_20943_b300 import RasterConfig, Rasterizer
    return Rasterizer(RasterConfig(sort_mode=0, cull_lists=False))


_by_shape = {}


def rast_shape(shape):
    """A context pinned to one compiled kernel shape (radix ordering, half-tile
    lists).  Shape 0 is the default; a shape index packs (forward f, backward
    b, sort k, emission e) as f + NF (b + NB (k + NS e)): the forward's and the
    backward's staging batch / warps per SM, the instance sort's keys per
    thread and the emission's instances per thread (Rasterizer.shape_names())."""
    from paper_2512_20943_b300 import RasterConfig, Rasterizer
    if shape not in _by_shape:
        _by_shape[shape] = Rasterizer(RasterConfig(kernel_shape=shape, sort_mode=0))
    return _by_shape[shape]


NF, NB, NS, NE = 5, 5, 3, 3      # compiled forward, backward, sort and emission shapes
FWD_SHAPES = list(range(NF))                       # forward (batch, warps) axis, the rest at shape 0
BWD_SHAPES = [NF * b for b in range(NB)]           # backward (batch, warps) axis
SORT_SHAPES = [NF * NB * k for k in range(NS)]     # instance-sort keys per thread axis
EMIT_SHAPES = [NF * NB * NS * e for e in range(NE)]  # emission instances-per-thread axis
SHAPES = sorted(set(FWD_SHAPES + BWD_SHAPES + SORT_SHAPES + EMIT_SHAPES))


def render_gpu(rast, g, cams, **kw):
    t = to_cuda(g)
    res = rast.render_gaussians(*params(t), cams, **kw)
    torch.cuda.synchronize()
    return t, res


def scenes():
    g1, c1 = synthetic.plain_forward_scene()
    g2, c2 = small_sh3_scene()
    return {"plain_2k": (g1, c1), "sh3_ragged": (g2, c2)}


@pytest.mark.parametrize("name", ["plain_2k", "sh3_ragged"])
def test_projection_matches_oracle(rast, name):
    g, cams = scenes()[name]
    t, res = render_gpu(rast, g, cams, save=True)
    for v, cam in enumerate(cams):
        m2, d, r = (x.cpu().numpy() for x in rast.state_projection(res.state, v))
        ref = oracle.project(synthetic.widen(g), cam)
        ok = (ref["ambig"] == 0) & (ref["visible"] == 1)
        assert ok.sum() > 0.5 * ref["visible"].sum()
        assert np.array_equal(r[ok], ref["radius"][ok])
        assert np.abs(m2[ok] - ref["mean2d"][ok]).max() < 1e-3
        assert np.abs(d[ok] - ref["depth"][ok]).max() < 1e-5 * np.abs(ref["depth"]).max()
        # culled exactly where the oracle culls
        unamb = ref["ambig"] == 0
        assert np.array_equal(r[unamb] > 0, ref["visible"][unamb] == 1)
    res.state.release()


_by_sort = {}


def rast_sort(mode):
    """A context pinned to an ordering path: 1 per-tile lists sorted in shared
    memory, 0 the global two-stage radix ordering (default); full lists."""
    from paper_2512_20943_b300 import RasterConfig, Rasterizer
    if mode not in _by_sort:
        _by_sort[mode] = Rasterizer(RasterConfig(sort_mode=mode, cull_lists=False))
    return _by_sort[mode]


@pytest.mark.parametrize("sort_mode", [1, 0])
@pytest.mark.parametrize("name", ["plain_2k", "sh3_ragged"])
def test_tile_lists_bit_exact(name, sort_mode):
    """The GPU's binning and stable (tile, depth, index) ordering equal the
    oracle's when the oracle is given the GPU's own centres, radii and depths."""
    rast = rast_sort(sort_mode)
    g, cams = scenes()[name]
    t, res = render_gpu(rast, g, cams, save=True)
    for v, cam in enumerate(cams):
        m2, d, r = (x.cpu().numpy() for x in rast.state_projection(res.state, v))
        ranges, ids = (x.cpu().numpy() for x in rast.state_tile_lists(res.state, v))
        ref_ranges, ref_ids = oracle.bin_sort(m2.astype(np.float64), r, d.astype(np.float64), r > 0, cam["width"],
                                              cam["height"])
        assert np.array_equal(ranges, ref_ranges)
        assert np.array_equal(ids, ref_ids)
        assert len(ids) > 0
    res.state.release()


@pytest.mark.parametrize("name", ["plain_2k", "sh3_ragged"])
def test_tile_lists_match_fp64_sets(rast, name):
    g, cams = scenes()[name]
    t, res = render_gpu(rast, g, cams, save=True)
    for v, cam in enumerate(cams):
        ranges, ids = (x.cpu().numpy() for x in rast.state_tile_lists(res.state, v))
        ref = oracle.project(synthetic.widen(g), cam)
        ref_ranges, ref_ids = oracle.bin_sort(ref["mean2d"], ref["radius"], ref["depth"], ref["visible"],
                                              cam["width"], cam["height"])
        amb = set(np.nonzero(ref["ambig"])[0].tolist())
        for tile in range(len(ranges)):
            a = [i for i in ids[ranges[tile, 0]:ranges[tile, 1]] if i not in amb]
            b = [i for i in ref_ids[ref_ranges[tile, 0]:ref_ranges[tile, 1]] if i not in amb]
            assert a == b, tile
    res.state.release()


@pytest.mark.parametrize("shape", sorted(set(FWD_SHAPES + SORT_SHAPES + EMIT_SHAPES)))
@pytest.mark.parametrize("name", ["plain_2k", "sh3_ragged"])
def test_forward_matches_oracle(name, shape):
    rast = rast_shape(shape)
    g, cams = scenes()[name]
    t, res = render_gpu(rast, g, cams, T=True, n_contrib=True)
    ref = oracle.render(synthetic.widen(g), cams)
    rgb, T, nc = views_np(res.rgb, cams), views_np(res.T, cams, 1), views_np(res.n_contrib, cams, 1)
    for v in range(len(cams)):
        ok = ~ref["ambig"][v]
        assert ok.mean() > 0.97
        assert np.abs(rgb[v] - ref["rgb"][v])[:, ok].max() < RGB_ATOL
        assert np.abs(T[v] - ref["T"][v])[ok].max() < RGB_ATOL
        assert np.array_equal(nc[v][ok], ref["n_contrib"][v][ok])
        assert (rgb[v] >= 0).all() and ((T[v] >= 0) & (T[v] <= 1)).all()
    assert max(r.max() for r in ref["rgb"]) > 0.2  # not an empty image


@pytest.mark.parametrize("shape", SHAPES)
def test_importance_matches_oracle(shape):
    rast = rast_shape(shape)
    g, cams = small_sh3_scene()
    t, res = render_gpu(rast, g, cams, importance=True, save=True)
    ref = oracle.render(synthetic.widen(g), cams)
    ok = ref["gauss_ambig"] == 0
    w = res.importance_w.cpu().numpy()
    c = res.importance_cnt.cpu().numpy()
    assert ok.mean() > 0.8
    assert np.array_equal(c[ok], ref["importance_cnt"][ok])
    assert np.abs(w - ref["importance_w"])[ok].max() < 1e-3 * max(1.0, ref["importance_w"].max())
    # the backward replay accumulates the same usage frequency
    iw = torch.zeros_like(res.importance_w)
    ic = torch.zeros_like(res.importance_cnt)
    rast.render_backward(res.state, torch.zeros_like(res.rgb), importance=(iw, ic))
    torch.cuda.synchronize()
    assert np.array_equal(ic.cpu().numpy(), c)
    assert np.abs(iw.cpu().numpy() - w).max() < 1e-4 * max(1.0, w.max())
    # gaussian_importance over the context's frame state
    rast.set_anchor(*params(t))
    w2, c2 = rast.gaussian_importance(cams)
    torch.cuda.synchronize()
    assert np.array_equal(c2.cpu().numpy(), c)
    res.state.release()


def masked_dL(cams, ref, seed):
    rng = np.random.default_rng(seed)
    out = []
    for v, c in enumerate(cams):
        d = rng.standard_normal((3, c["height"], c["width"]))
        d[:, ref["ambig"][v]] = 0.0  # no loss on pixels with a near-threshold decision
        out.append(d)
    return out


@pytest.mark.parametrize("shape", BWD_SHAPES)
@pytest.mark.parametrize("name", ["plain_2k", "sh3_ragged"])
def test_backward_matches_oracle(name, shape):
    rast = rast_shape(shape)
    g, cams = scenes()[name]
    ref = oracle.render(synthetic.widen(g), cams)
    dL = masked_dL(cams, ref, 5)
    t, res = render_gpu(rast, g, cams, save=True)
    flat = torch.from_numpy(np.concatenate([d.reshape(-1) for d in dL]).astype(np.float32)).cuda()
    gr = rast.render_backward(res.state, flat)
    torch.cuda.synchronize()
    ref_g = oracle.render_backward(synthetic.widen(g), cams, dL)
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        assert_grad_close(gr[k].cpu().numpy(), ref_g[k], k)
    res.state.release()


@pytest.mark.parametrize("shape", BWD_SHAPES)
def test_l1_fused_equals_explicit_gradient(shape):
    rast = rast_shape(shape)
    g, cams = small_sh3_scene()
    tgt = synthetic.target_images(cams, 1)
    target = torch.from_numpy(np.concatenate([x.reshape(-1) for x in tgt])).cuda()
    t, res = render_gpu(rast, g, cams, save=True)
    loss, gr = rast.render_backward_l1(res.state, target)
    n = res.rgb.numel()
    dL = torch.sign(res.rgb - target) / n
    gr2 = rast.render_backward(res.state, dL.contiguous())
    torch.cuda.synchronize()
    ref_loss = float(torch.abs(res.rgb.double() - target.double()).mean())
    assert abs(float(loss) - ref_loss) < 1e-5 * ref_loss
    for k in gr:
        a, b = gr[k].cpu().numpy(), gr2[k].cpu().numpy()
        assert np.abs(a - b).max() <= 1e-5 * max(np.abs(b).max(), 1e-30), k
    # and against the oracle's L1 definition
    ref = oracle.render(synthetic.widen(g), cams)
    ref_loss2, _ = oracle.l1_loss_grad(ref["rgb"], [x.astype(np.float64) for x in tgt])
    assert abs(float(loss) - ref_loss2) < 1e-4
    res.state.release()


def test_decode_apply_matches_oracle(rast):
    N = 3000
    g = synthetic.gaussians(N, 3, sh_degree=1)
    t = to_cuda(g)
    rast.set_anchor(*params(t))
    m1, lo, hi = synthetic.update_map(N, 1001, size=64)
    m2, _, _ = synthetic.update_map(N, 1002, size=64)
    for mode_name in ("prev", "anchor", "add"):
        rast.set_anchor(*params(t))
        from paper_2512_20943_b300 import AIRGS_DELTA_ANCHOR, AIRGS_DELTA_PREV
        mode = AIRGS_DELTA_ANCHOR if mode_name == "anchor" else AIRGS_DELTA_PREV
        qa = mode_name == "add"
        rast.apply_frame_update(torch.from_numpy(m1.view(np.int16)).cuda().view(torch.uint16), lo, hi, mode=mode,
                                quat_add=qa)
        rast.apply_frame_update(torch.from_numpy(m2.view(np.int16)).cuda().view(torch.uint16), lo, hi, mode=mode,
                                quat_add=qa)
        means, quats = (x.cpu().numpy() for x in rast.frame_state())
        w = synthetic.widen(g)
        qm = oracle.QUAT_ADD if qa else oracle.QUAT_COMPOSE
        lo64, hi64 = lo.astype(np.float64), hi.astype(np.float64)
        if mode_name == "anchor":
            rm, rq = oracle.decode_apply(m2, lo64, hi64, w["means"], w["quats"], qm)
        else:
            am, aq = oracle.decode_apply(m1, lo64, hi64, w["means"], w["quats"], qm)
            rm, rq = oracle.decode_apply(m2, lo64, hi64, am, aq, qm)
        assert np.abs(means - rm).max() < 2e-6 * max(1, np.abs(rm).max())
        assert np.abs(quats - rq).max() < 2e-6


@pytest.mark.parametrize("n,bits", [(1, 8), (4095, 13), (4096, 32), (4097, 16), (1_000_003, 24), (3_000_000, 32)])
def test_radix_sort_stable_bit_exact(rast, n, bits):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 1 << min(bits, 20), n, dtype=np.uint64).astype(np.uint32)  # many duplicates
    if bits > 20:
        keys = (keys.astype(np.uint64) << np.uint64(bits - 20)).astype(np.uint32)
    vals = np.arange(n, dtype=np.uint32)
    kt = torch.from_numpy(keys.view(np.int32)).cuda()
    vt = torch.from_numpy(vals.view(np.int32)).cuda()
    ko, vo = rast.sort_pairs(kt, vt, bits)
    torch.cuda.synchronize()
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(ko.cpu().numpy().view(np.uint32), keys[order])
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), vals[order])


@pytest.mark.parametrize("n,bits", [(200_003, 17), (65_537, 5), (100_000, 30)])
def test_radix_sort_ignores_bits_above_key_bits(rast, n, bits):
    """Only bits [0, key_bits) order the pairs (the tile sort keeps flags in the
    top bits of its keys); the keys come out whole."""
    rng = np.random.default_rng(n + bits)
    keys = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    vals = np.arange(n, dtype=np.uint32)
    ko, vo = rast.sort_pairs(torch.from_numpy(keys.view(np.int32)).cuda(),
                             torch.from_numpy(vals.view(np.int32)).cuda(), bits)
    torch.cuda.synchronize()
    order = np.argsort(keys & np.uint32((1 << bits) - 1), kind="stable")
    assert np.array_equal(ko.cpu().numpy().view(np.uint32), keys[order])
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), vals[order])


@pytest.mark.parametrize("shape", [0, 2, 50])
def test_permutation_invariance_gpu(shape):
    rast = rast_shape(shape)
    g, cams = small_sh3_scene()
    perm = np.random.default_rng(4).permutation(g["means"].shape[0])
    gp = dict(g)
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        gp[k] = np.ascontiguousarray(g[k][perm])
    _, a = render_gpu(rast, g, cams)
    _, b = render_gpu(rast, gp, cams)
    # same lists up to relabelling, same arithmetic: identical images
    assert torch.equal(a.rgb, b.rgb)


def test_degenerate_inputs(rast):
    from paper_2512_20943_b300 import AirGSError
    # no Gaussians
    g = synthetic.gaussians(0, 0, sh_degree=0)
    cams = [synthetic.camera((0, 0, -4.0), 40, 30, fov_x_deg=60)]
    _, res = render_gpu(rast, g, cams, T=True)
    assert float(res.rgb.abs().max()) == 0.0 and float(res.T.min()) == 1.0
    # everything behind the camera
    g = synthetic.gaussians(50, 1, sh_degree=0)
    g["means"][:, 2] = -10.0
    _, res = render_gpu(rast, g, cams, T=True)
    assert float(res.rgb.abs().max()) == 0.0
    # a 1x1 image and a 17x1 strip
    g = synthetic.gaussians(200, 2, mean_mode="uniform", mean_scale=(1, 1, 1), log_scale=(-2.5, 0.3), sh_degree=0)
    cams = [synthetic.camera((0, 0, -4.0), 1, 1, fx=1.0), synthetic.camera((0, 0, -4.0), 17, 1, fx=17.0)]
    _, res = render_gpu(rast, g, cams)
    ref = oracle.render(synthetic.widen(g), cams)
    rgb = views_np(res.rgb, cams)
    for v in range(2):
        ok = ~ref["ambig"][v]
        assert np.abs(rgb[v] - ref["rgb"][v])[:, ok].max() < RGB_ATOL
    # argument errors are reported, not crashed on
    with pytest.raises(AirGSError):
        rast.render_gaussians(*params(to_cuda(g)), [])


def test_frame_update_map_too_small_is_an_error(rast):
    from paper_2512_20943_b300 import AirGSError
    g = synthetic.gaussians(100, 0, sh_degree=0)
    rast.set_anchor(*params(to_cuda(g)))
    with pytest.raises(AirGSError):
        rast.apply_frame_update(torch.zeros((7, 5, 5), dtype=torch.uint16, device="cuda"), np.zeros(7), np.ones(7))


def needle_scene(thin=-7.0, long=-1.5):
    """Needle-like and sub-pixel Gaussians (one log-scale near `thin`, another
    near `long`), opaque and faint, many near the alpha_min ellipse of each
    culling block: the case where block culling by bounding box or by ellipse
    is tightest.  Long needles have screen-space conics whose determinant
    cancels to about 1e-3 of their entries, beyond what single-precision
    gradients can match to 1e-3, so the gradient test uses shorter ones."""
    g = synthetic.gaussians(3000, 77, mean_mode="uniform", mean_scale=(1.5, 1.2, 1.0), log_scale=(-4.0, 1.5),
                            sh_degree=1, opacity_std=3.0)
    rng = np.random.default_rng(78)
    ls = g["log_scales"]
    ls[:, 0] = rng.normal(thin, 0.5, ls.shape[0])
    ls[:, 1] = rng.normal(long, 0.5, ls.shape[0])
    cams = [synthetic.camera((0.1, 0.0, -4.0), 160, 120, fov_x_deg=55.0),
            synthetic.camera((1.5, -0.5, -3.5), 97, 61, fov_x_deg=40.0)]
    return g, cams


def test_autotune_chooses_a_shape_and_round_trips_its_cache(tmp_path):
    """The autotuner times training steps over the compiled shapes (shape 0
    included, so the choice is not slower than it), later renders of the same
    workload run the choice, and a new context reads it back from the cache."""
    from paper_2512_20943_b300 import RasterConfig, Rasterizer
    path = tmp_path / "shapes.txt"
    g, cams = small_sh3_scene()
    t = to_cuda(g)
    rast = Rasterizer(RasterConfig(autotune_cache=str(path)))
    rast.set_anchor(*params(t))
    res = rast.render(cams, save=True)
    assert rast.stats(res.state)["kernel_shape"] == 0  # untuned: the default shape
    res.state.release()
    shape, ms_default, ms_best = rast.autotune(cams, report=True)
    assert 0 <= shape < len(Rasterizer.shape_names())
    assert 0.0 < ms_best <= ms_default
    res = rast.render(cams, save=True)
    assert rast.stats(res.state)["kernel_shape"] == shape
    res.state.release()
    lines = path.read_text().split()
    assert lines[-1] == str(shape)
    again = Rasterizer(RasterConfig(autotune_cache=str(path)))
    again.set_anchor(*params(t))
    res = again.render(cams, save=True)
    assert again.stats(res.state)["kernel_shape"] == shape
    res.state.release()
    # a pinned shape wins over the tuned one
    pinned = Rasterizer(RasterConfig(autotune_cache=str(path), kernel_shape=3))
    pinned.set_anchor(*params(t))
    res = pinned.render(cams, save=True)
    assert pinned.stats(res.state)["kernel_shape"] == 3
    res.state.release()


@pytest.mark.parametrize("scene", ["sh3_ragged", "needles", "thin_needles"])
def test_shapes_agree(scene):
    """Every kernel shape evaluates the same pairs with the same arithmetic:
    images, transmittance, n_contrib and blended-pair counts are bit-identical
    across shapes.  Gradients differ only in the order of the atomic additions
    into each Gaussian's record, which the needle scene's ill-conditioned
    log-scale gradients amplify to about 1e-3 between any two runs, so every
    shape's gradients are held to the oracle's (loss off the flagged pixels);
    the thinnest needles (log-scale -7, where culling is tightest) are compared
    in the forward only."""
    if scene == "sh3_ragged":
        g, cams = small_sh3_scene()
    else:
        g, cams = needle_scene(thin=-3.5, long=-2.0) if scene == "needles" else needle_scene()
    grads = scene != "thin_needles"
    ref = oracle.render(synthetic.widen(g), cams)
    dL = masked_dL(cams, ref, 77)
    flat = torch.from_numpy(np.concatenate([d.reshape(-1) for d in dL]).astype(np.float32)).cuda()
    ref_g = oracle.render_backward(synthetic.widen(g), cams, dL) if grads else None
    outs = []
    for shp in SHAPES:
        rast = rast_shape(shp)
        _, o = render_gpu(rast, g, cams, T=True, n_contrib=True, importance=True, save=True)
        gr = rast.render_backward(o.state, flat)
        torch.cuda.synchronize()
        assert rast.stats(o.state)["kernel_shape"] == shp
        for k in ("means", "log_scales", "quats", "opacity_logit", "sh") if grads else ():
            assert_grad_close(gr[k].cpu().numpy(), ref_g[k], (shp, k))
        outs.append(o)
        o.state.release()
    o0 = outs[0]
    for o in outs[1:]:
        assert torch.equal(o.rgb, o0.rgb)
        assert torch.equal(o.T, o0.T)
        assert torch.equal(o.n_contrib, o0.n_contrib)
        assert torch.equal(o.importance_cnt, o0.importance_cnt)
    assert int(o0.importance_cnt.sum()) > 0


def large_faint_scene():
    """A few dozen large, faint Gaussians: each covers whole 16x16 tiles with
    every pixel blending it (an entry's 128 pixels of a half tile all blended,
    the count's largest value per entry) and no pixel saturates."""
    g = synthetic.gaussians(24, 5, mean_mode="uniform", mean_scale=(0.6, 0.5, 0.3), log_scale=(-0.9, 0.15),
                            sh_degree=1)
    g["opacity_logit"][:] = -2.0
    cams = [synthetic.camera((0.0, 0.0, -4.0), 100, 70, fov_x_deg=50.0),
            synthetic.camera((0.4, -0.3, -3.6), 53, 37, fov_x_deg=55.0)]
    return g, cams


@pytest.mark.parametrize("shape", [0, 10])
def test_large_gaussians_backward_counts_and_gradients(shape):
    """Usage counts accumulated by the backward replay equal the forward's
    (and the oracle's) when every entry blends whole tiles, and the gradients
    match the oracle's."""
    rast = rast_shape(shape)
    g, cams = large_faint_scene()
    ref = oracle.render(synthetic.widen(g), cams)
    t, res = render_gpu(rast, g, cams, importance=True, save=True)
    c = res.importance_cnt.cpu().numpy()
    assert c.max() > 2 * 256  # several full tiles per Gaussian
    ok = ref["gauss_ambig"] == 0
    assert np.array_equal(c[ok], ref["importance_cnt"][ok])
    iw = torch.zeros_like(res.importance_w)
    ic = torch.zeros_like(res.importance_cnt)
    dL = masked_dL(cams, ref, 31)
    flat = torch.from_numpy(np.concatenate([d.reshape(-1) for d in dL]).astype(np.float32)).cuda()
    gr = rast.render_backward(res.state, flat, importance=(iw, ic))
    torch.cuda.synchronize()
    assert np.array_equal(ic.cpu().numpy(), c)
    w = res.importance_w.cpu().numpy()
    assert np.abs(iw.cpu().numpy() - w).max() < 1e-4 * max(1.0, w.max())
    ref_g = oracle.render_backward(synthetic.widen(g), cams, dL)
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        assert_grad_close(gr[k].cpu().numpy(), ref_g[k], k)
    res.state.release()


def clamped_scene():
    """Twelve opaque (o = 0.9975), wide Gaussians in front of a faint layer: in
    20 of their 24 (view, Gaussian) projections some pixel has o G above
    alpha_max = 0.99, so the replay meets clamped pairs (alpha = alpha_max, no
    gradient to o or G) next to unclamped ones."""
    g = synthetic.gaussians(150, 41, mean_mode="uniform", mean_scale=(1.3, 1.0, 0.8), log_scale=(-3.0, 0.4),
                            sh_degree=1)
    rng = np.random.default_rng(42)
    g["opacity_logit"][:] = rng.normal(-1.0, 0.7, 150)
    g["opacity_logit"][:12] = 6.0
    g["log_scales"][:12] = rng.normal(-1.6, 0.15, (12, 3))
    g["means"][:12, 2] -= 0.6
    cams = [synthetic.camera((0.0, 0.0, -4.0), 96, 72, fov_x_deg=50.0),
            synthetic.camera((0.5, 0.3, -3.8), 61, 45, fov_x_deg=55.0)]
    return g, cams


@pytest.mark.parametrize("shape", [0, 10])
def test_clamped_alpha_gradients_match_oracle(shape):
    """Gradients through pairs whose alpha is clamped at alpha_max (the replay
    tells them from unclamped ones by ae == o G) match the oracle's."""
    rast = rast_shape(shape)
    g, cams = clamped_scene()
    ref = oracle.render(synthetic.widen(g), cams)
    dL = masked_dL(cams, ref, 43)
    t, res = render_gpu(rast, g, cams, save=True)
    flat = torch.from_numpy(np.concatenate([d.reshape(-1) for d in dL]).astype(np.float32)).cuda()
    gr = rast.render_backward(res.state, flat)
    torch.cuda.synchronize()
    ref_g = oracle.render_backward(synthetic.widen(g), cams, dL)
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        assert_grad_close(gr[k].cpu().numpy(), ref_g[k], k)
    res.state.release()


@pytest.mark.parametrize("shape", [0, 10])
def test_needles_backward_matches_oracle(shape):
    rast = rast_shape(shape)
    g, cams = needle_scene(thin=-3.5, long=-2.0)
    ref = oracle.render(synthetic.widen(g), cams)
    dL = masked_dL(cams, ref, 9)
    t, res = render_gpu(rast, g, cams, save=True)
    assert np.abs(views_np(res.rgb, cams)[0] - ref["rgb"][0])[:, ~ref["ambig"][0]].max() < RGB_ATOL
    flat = torch.from_numpy(np.concatenate([d.reshape(-1) for d in dL]).astype(np.float32)).cuda()
    gr = rast.render_backward(res.state, flat)
    torch.cuda.synchronize()
    ref_g = oracle.render_backward(synthetic.widen(g), cams, dL)
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        assert_grad_close(gr[k].cpu().numpy(), ref_g[k], k)
    res.state.release()


@pytest.mark.parametrize("n", [5000, 20000])
def test_long_tile_lists(n):
    """Lists longer than one 256-thread CTA sorts (5000 entries: the 1024-thread
    path) and longer than one CTA can hold (20000: the global radix fallback)
    are ordered exactly like the oracle's."""
    rng = np.random.default_rng(n)
    g = synthetic.gaussians(n, n, mean_mode="uniform", mean_scale=(0.02, 0.02, 1.0), log_scale=(-4.5, 0.3),
                            sh_degree=0, rgb_dc=True)
    g["opacity_logit"][:] = -3.0  # faint, so pixels do not stop early
    cams = [synthetic.camera((0, 0, -4.0), 32, 32, fx=32.0)]
    rast = rast_sort(1)
    t, res = render_gpu(rast, g, cams, save=True)
    m2, d, r = (x.cpu().numpy() for x in rast.state_projection(res.state, 0))
    ranges, ids = (x.cpu().numpy() for x in rast.state_tile_lists(res.state, 0))
    ref_ranges, ref_ids = oracle.bin_sort(m2.astype(np.float64), r, d.astype(np.float64), r > 0, 32, 32)
    assert (ranges[:, 1] - ranges[:, 0]).max() > (4096 if n > 10000 else 2048)
    assert np.array_equal(ranges, ref_ranges)
    assert np.array_equal(ids, ref_ids)
    ref = oracle.render(synthetic.widen(g), cams)
    ok = ~ref["ambig"][0]
    assert np.abs(views_np(res.rgb, cams)[0] - ref["rgb"][0])[:, ok].max() < RGB_ATOL
    res.state.release()


def test_densify_statistics_match_oracle():
    """Sum over views of |dL/d mean2d| and the visible-view count per Gaussian
    (densification statistics of keyframe reconstruction), and the selection."""
    from paper_2512_20943_b300 import Rasterizer
    rast = Rasterizer()
    g, cams = small_sh3_scene()
    ref = oracle.render(synthetic.widen(g), cams)
    dL = masked_dL(cams, ref, 8)
    t, res = render_gpu(rast, g, cams, save=True)
    n = g["means"].shape[0]
    dg = torch.zeros(n, dtype=torch.float32, device="cuda")
    dv = torch.zeros(n, dtype=torch.int32, device="cuda")
    flat = torch.from_numpy(np.concatenate([d.reshape(-1) for d in dL]).astype(np.float32)).cuda()
    rast.render_backward_ex(res.state, dL_drgb=flat, densify=(dg, dv))
    torch.cuda.synchronize()
    ref_g = oracle.render_backward(synthetic.widen(g), cams, dL, densify=True)
    ok = ref["gauss_ambig"] == 0
    assert np.array_equal(dv.cpu().numpy()[ok], ref_g["densify_views"][ok])
    assert_grad_close(dg.cpu().numpy()[ok], ref_g["densify_grad"][ok], "densify_grad")
    thr = float(np.median(ref_g["densify_grad"][ref_g["densify_views"] > 0] /
                          ref_g["densify_views"][ref_g["densify_views"] > 0]))
    mask = rast.densify_select(dg, dv, thr).cpu().numpy()
    d, v = dg.cpu().numpy(), dv.cpu().numpy()
    assert np.array_equal(mask, ((v > 0) & (d > thr * v)).astype(np.uint8))
    assert 0 < mask.sum() < n
    res.state.release()


def test_fp32_probe_reports_a_plausible_peak(rast):
    """The FMA probe the benchmark reports beside the derived FP32 peak."""
    v = rast.measure_fp32_peak()
    assert 10.0 < v < 200.0, v


def test_smem_probe_reports_a_plausible_peak(rast):
    """The shared-memory load probe the benchmark reports beside the derived
    shared-memory peak (SMs x 128 B per clock): within a factor of two of it."""
    v = rast.measure_smem_peak()
    props = torch.cuda.get_device_properties(0)
    derived = props.multi_processor_count * 128 * 2.0e9 / 1e12  # at about 2 GHz
    assert 0.5 * derived < v < 2.0 * derived, (v, derived)


@pytest.mark.parametrize("scene", ["plain_2k", "sh3_ragged", "needles", "dense_cluster"])
def test_culled_lists_render_identically(scene):
    """Renders that do not return n_contrib list a Gaussian only in tiles where
    it can reach alpha_min -- the tiles its ellipse's exact row bands meet when
    no state is kept, the tiles its bounding box meets for a state saved for a
    backward: images, transmittance and blended-pair counts are bit-identical
    to the full rectangle lists, with the default and another forward shape,
    with fewer list entries; the backward of a saved state replays its culled
    lists and gives the full lists' usage counts exactly and their gradients
    within the gradient bar (only the order of the atomic additions differs;
    the thinnest needles' ill-conditioned log-scale gradients amplify that
    order to about 1e-3, so that scene is compared in the forward only)."""
    from paper_2512_20943_b300 import RasterConfig, Rasterizer
    if scene == "needles":
        g, cams = needle_scene()
    elif scene == "dense_cluster":  # the serving workload's shape, scaled down
        g = synthetic.serving_scene(20000, seed=3)
        rng = np.random.default_rng(11)
        cams = [synthetic.camera(synthetic.sphere_pose(rng, 3.0), w, h, fov_x_deg=60.0)
                for (w, h) in [(320, 240), (200, 113), (480, 270)]]
    else:
        g, cams = scenes()[scene]
    rng = np.random.default_rng(5)
    for v in (0, 2):
        full = Rasterizer(RasterConfig(kernel_shape=v, cull_lists=False, sort_mode=0))
        culled = Rasterizer(RasterConfig(kernel_shape=v, cull_lists=True, sort_mode=0))
        bands = render_gpu(culled, g, cams, T=True, importance=True)[1]  # no state: the exact row bands
        a = render_gpu(full, g, cams, T=True, importance=True, save=True)[1]
        b = render_gpu(culled, g, cams, T=True, importance=True, save=True)[1]  # saved: the alpha_min box
        assert torch.equal(a.rgb, bands.rgb) and torch.equal(a.T, bands.T), v
        assert torch.equal(a.importance_cnt, bands.importance_cnt), v
        assert torch.equal(a.rgb, b.rgb), v
        assert torch.equal(a.T, b.T), v
        assert torch.equal(a.importance_cnt, b.importance_cnt), v
        assert float(a.rgb.max()) > 0.0
        assert culled.stats(b.state)["n_instances"] < full.stats(a.state)["n_instances"]
        dL = torch.from_numpy(rng.standard_normal(a.rgb.numel()).astype(np.float32)).cuda()
        ia = (torch.zeros_like(a.importance_w), torch.zeros_like(a.importance_cnt))
        ib = (torch.zeros_like(b.importance_w), torch.zeros_like(b.importance_cnt))
        ga = full.render_backward(a.state, dL, importance=ia)
        gb = culled.render_backward(b.state, dL, importance=ib)
        torch.cuda.synchronize()
        assert torch.equal(ia[1], ib[1]) and torch.equal(ib[1], a.importance_cnt), v
        if scene != "needles":
            for k in ga:
                assert_grad_close(gb[k].cpu().numpy(), ga[k].cpu().numpy(), (v, k))
        a.state.release()
        b.state.release()


@pytest.mark.gpu
def test_unaligned_sh_buffer_renders_identically(rast):
    """The projection reads SH coefficients with 16-byte loads only from a
    16-byte aligned buffer; a buffer that starts 4 bytes off takes the scalar
    path and must give bit-identical images and gradients."""
    g, cams = small_sh3_scene()
    t = to_cuda(g)
    p = list(params(t))
    sh = p[4]
    store = torch.empty(sh.numel() + 4, dtype=torch.float32, device=sh.device)
    shifted = store[1:1 + sh.numel()].view(sh.shape)
    shifted.copy_(sh)
    assert shifted.data_ptr() % 16 != 0 and sh.data_ptr() % 16 == 0
    a = rast.render_gaussians(*p, cams, save=True)
    b = rast.render_gaussians(*p[:4], shifted, cams, save=True)
    assert torch.equal(a.rgb, b.rgb)
    dL = torch.ones_like(a.rgb)
    ga = {k: v.clone() for k, v in rast.render_backward(a.state, dL).items()}
    gb = rast.render_backward(b.state, dL)
    # gradients are accumulated with atomics, so they agree up to the order of the
    # additions; held to the parity bars of the gradient tests
    for k in ga:
        assert_grad_close(gb[k].cpu().numpy(), ga[k].cpu().numpy(), k)
    a.state.release()
    b.state.release()


@pytest.mark.parametrize("shape", [0, 1])
def test_many_ragged_views_in_one_launch(shape):
    """40 views of sizes from 1x1 to 61x43 pixels (most not multiples of the
    16-pixel tile) and random poses, rendered and back-propagated in one
    launch: every view matches the oracle (each (view, tile) item finds its
    view among the 40 tile bases)."""
    rast = rast_shape(shape)
    g = synthetic.gaussians(600, 31, mean_mode="uniform", mean_scale=(1.0, 1.0, 1.0), log_scale=(-3.0, 0.5),
                            sh_degree=2, sh_std=0.2)
    rng = np.random.default_rng(32)
    sizes = [(1, 1), (61, 43), (16, 16), (17, 15)] + [(int(rng.integers(1, 62)), int(rng.integers(1, 44)))
                                                      for _ in range(36)]
    cams = [synthetic.camera(synthetic.sphere_pose(rng, 3.5), w, h, fov_x_deg=55.0) for (w, h) in sizes]
    ref = oracle.render(synthetic.widen(g), cams)
    t, res = render_gpu(rast, g, cams, T=True, save=True)
    rgb, T = views_np(res.rgb, cams), views_np(res.T, cams, 1)
    for v in range(len(cams)):
        ok = ~ref["ambig"][v]
        if ok.any():
            assert np.abs(rgb[v] - ref["rgb"][v])[:, ok].max() < RGB_ATOL, v
            assert np.abs(T[v] - ref["T"][v])[ok].max() < RGB_ATOL, v
    assert max(r.max() for r in ref["rgb"]) > 0.1
    dL = masked_dL(cams, ref, 33)
    flat = torch.from_numpy(np.concatenate([d.reshape(-1) for d in dL]).astype(np.float32)).cuda()
    gr = rast.render_backward(res.state, flat)
    torch.cuda.synchronize()
    ref_g = oracle.render_backward(synthetic.widen(g), cams, dL)
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        assert_grad_close(gr[k].cpu().numpy(), ref_g[k], k)
    res.state.release()


def test_maximum_view_count(rast):
    """AIRGS_MAX_VIEWS (256) views render in one launch and match the oracle;
    one more is an argument error."""
    from paper_2512_20943_b300 import AirGSError
    from paper_2512_20943_b300._abi import AIRGS_MAX_VIEWS
    g = synthetic.gaussians(300, 41, mean_mode="uniform", mean_scale=(1.0, 1.0, 1.0), log_scale=(-2.5, 0.4),
                            sh_degree=1, sh_std=0.2)
    rng = np.random.default_rng(42)
    cams = [synthetic.camera(synthetic.sphere_pose(rng, 3.5), 9 + v % 8, 7 + v % 5, fov_x_deg=50.0)
            for v in range(AIRGS_MAX_VIEWS)]
    t, res = render_gpu(rast, g, cams, T=True)
    ref = oracle.render(synthetic.widen(g), cams)
    rgb = views_np(res.rgb, cams)
    for v in range(len(cams)):
        ok = ~ref["ambig"][v]
        if ok.any():
            assert np.abs(rgb[v] - ref["rgb"][v])[:, ok].max() < RGB_ATOL, v
    assert max(r.max() for r in ref["rgb"]) > 0.1
    with pytest.raises(AirGSError):
        rast.render_gaussians(*params(t), cams + cams[:1])


@pytest.mark.parametrize("shape", [0, 15])
def test_non_default_settings_match_oracle(shape):
    """A coloured background, no low-pass dilation and other blending
    thresholds (alpha clamp 0.9, skip below 0.01, stop below 1e-3), on the GPU
    and in the oracle: images, T, n_contrib and gradients (the background
    enters the colour still ahead of every pair)."""
    from paper_2512_20943_b300 import RasterConfig, Rasterizer
    st = dict(dilation=0.0, alpha_max=0.9, alpha_min=0.01, T_min=1e-3, bg=(0.2, 0.5, 0.9))
    rast = Rasterizer(RasterConfig(kernel_shape=shape, **st))
    g, cams = small_sh3_scene()
    ref = oracle.render(synthetic.widen(g), cams, **st)
    t, res = render_gpu(rast, g, cams, T=True, n_contrib=True, save=True)
    rgb, T, nc = views_np(res.rgb, cams), views_np(res.T, cams, 1), views_np(res.n_contrib, cams, 1)
    for v in range(len(cams)):
        ok = ~ref["ambig"][v]
        assert ok.mean() > 0.97
        assert np.abs(rgb[v] - ref["rgb"][v])[:, ok].max() < RGB_ATOL
        assert np.abs(T[v] - ref["T"][v])[ok].max() < RGB_ATOL
        assert np.array_equal(nc[v][ok], ref["n_contrib"][v][ok])
        assert rgb[v].min() >= 0.2 * T[v].min() - 1e-6  # the background shows through
    dL = masked_dL(cams, ref, 51)
    flat = torch.from_numpy(np.concatenate([d.reshape(-1) for d in dL]).astype(np.float32)).cuda()
    gr = rast.render_backward(res.state, flat)
    torch.cuda.synchronize()
    ref_g = oracle.render_backward(synthetic.widen(g), cams, dL, **st)
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        assert_grad_close(gr[k].cpu().numpy(), ref_g[k], k)
    res.state.release()


def test_autograd_function_gradients_match_oracle(rast):
    """The torch.autograd.Function around the library: a random linear loss of
    the rendered images back-propagated by autograd gives the oracle's
    gradients with respect to every raw parameter."""
    from paper_2512_20943_b300 import rasterize
    g, cams = small_sh3_scene()
    t = to_cuda(g)
    p = [x.clone().requires_grad_(True) for x in params(t)]
    rgb = rasterize(rast, *p, cams)
    ref = oracle.render(synthetic.widen(g), cams)
    dL = masked_dL(cams, ref, 61)
    w = torch.from_numpy(np.concatenate([d.reshape(-1) for d in dL]).astype(np.float32)).cuda()
    (rgb * w).sum().backward()
    ref_g = oracle.render_backward(synthetic.widen(g), cams, dL)
    for name, x in zip(("means", "log_scales", "quats", "opacity_logit", "sh"), p):
        assert x.grad is not None and x.grad.shape == x.shape, name
        assert_grad_close(x.grad.cpu().numpy(), ref_g[name], name)


@pytest.mark.parametrize("shape", [0, 20])
def test_small_batch_default_ordering_equals_radix(shape):
    """The default ordering (sort_mode -1) sorts small batches per tile in
    shared memory, with instance arrays sized by an upper bound (the render
    does not wait for the count): images, T, n_contrib, importance, the
    instance count and gradients equal the radix ordering's (tile lists are
    identical, so the blend is too)."""
    from paper_2512_20943_b300 import RasterConfig, Rasterizer
    g, cams = small_sh3_scene()
    out, n_inst = [], []
    for mode in (-1, 0):
        r = Rasterizer(RasterConfig(kernel_shape=shape, sort_mode=mode))
        t, res = render_gpu(r, g, cams, T=True, n_contrib=True, importance=True, save=True)
        gr = r.render_backward(res.state, torch.ones_like(res.rgb))
        torch.cuda.synchronize()
        n_inst.append(r.stats(res.state)["n_instances"])
        out.append((res, {k: v.clone() for k, v in gr.items()}))
    assert n_inst[0] == n_inst[1] > 0
    (a, ga), (b, gb) = out
    assert torch.equal(a.rgb, b.rgb) and torch.equal(a.T, b.T) and torch.equal(a.n_contrib, b.n_contrib)
    assert torch.equal(a.importance_cnt, b.importance_cnt)
    for k in ga:  # atomics: equal up to the order of the additions
        assert_grad_close(ga[k].cpu().numpy(), gb[k].cpu().numpy(), k)
    a.state.release()
    b.state.release()


def test_profiling_levels():
    """Level 1 brackets every stage, level 2 (the benchmark's timed region) only
    the two blend stages; both count the blend kernels' pairs; off times
    nothing; any other level is an argument error."""
    from paper_2512_20943_b300 import AirGSError, RasterConfig, Rasterizer
    rast = Rasterizer(RasterConfig(sort_mode=0))
    g, cams = small_sh3_scene()
    t = to_cuda(g)

    def step():
        res = rast.render_gaussians(*params(t), cams, save=True)
        rast.render_backward(res.state, torch.ones_like(res.rgb))
        res.state.release()
        return rast.stage_times()

    for level in ("all", "blend"):
        rast.set_profiling(True, blend_only=level == "blend")
        rast.stage_times()
        st = step()
        timed = {k for k, v in st["launches"].items() if v}
        if level == "blend":
            assert timed == {"blend_fwd", "blend_bwd"}
        else:
            assert {"project_sh", "depth_sort", "scan_emit", "tile_sort", "blend_fwd", "blend_bwd",
                    "project_bwd"} <= timed
        assert all(st["ms"][k] > 0 for k in timed)
        assert st["pairs_forward"] > 0 and st["pairs_backward"] > 0
    rast.set_profiling(False)
    rast.stage_times()
    st = step()
    assert not any(st["launches"].values()) and st["pairs_forward"] == 0
    with pytest.raises(AirGSError):
        rast._check(rast.lib.airgs_set_profiling(rast.ctx, 3))


_default_ordering = {}


@pytest.mark.parametrize("seed", range(8))
def test_random_scene_sweep(seed):
    """Seeded random scenes (1-2500 Gaussians, SH degree 0-3, scale and opacity
    spreads, 1-4 cameras of random sizes and poses), alternating the radix and
    the default ordering: image, T and n_contrib on unflagged pixels, exact
    blended-pair counts on unflagged Gaussians, and gradients vs the oracle."""
    from paper_2512_20943_b300 import Rasterizer
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(1, 2500))
    g = synthetic.gaussians(n, 2000 + seed, mean_mode="uniform", mean_scale=(1.2, 1.0, 1.2),
                            log_scale=(float(rng.uniform(-4.0, -2.2)), float(rng.uniform(0.2, 0.8))),
                            sh_degree=int(rng.integers(0, 4)), sh_std=0.2, opacity_std=float(rng.uniform(0.5, 2.5)))
    cams = [synthetic.camera(synthetic.sphere_pose(rng, float(rng.uniform(2.5, 4.5))), int(rng.integers(1, 161)),
                             int(rng.integers(1, 121)), fov_x_deg=float(rng.uniform(40.0, 70.0)))
            for _ in range(int(rng.integers(1, 5)))]
    if seed % 2:
        rast = _default_ordering.setdefault("ctx", Rasterizer())
    else:
        rast = rast_shape(0)
    ref = oracle.render(synthetic.widen(g), cams)
    t, res = render_gpu(rast, g, cams, T=True, n_contrib=True, importance=True, save=True)
    rgb, T, nc = views_np(res.rgb, cams), views_np(res.T, cams, 1), views_np(res.n_contrib, cams, 1)
    for v in range(len(cams)):
        ok = ~ref["ambig"][v]
        if ok.any():
            assert np.abs(rgb[v] - ref["rgb"][v])[:, ok].max() < RGB_ATOL, v
            assert np.abs(T[v] - ref["T"][v])[ok].max() < RGB_ATOL, v
            assert np.array_equal(nc[v][ok], ref["n_contrib"][v][ok]), v
    okg = ref["gauss_ambig"] == 0
    assert np.array_equal(res.importance_cnt.cpu().numpy()[okg], ref["importance_cnt"][okg])
    dL = masked_dL(cams, ref, 3000 + seed)
    flat = torch.from_numpy(np.concatenate([d.reshape(-1) for d in dL]).astype(np.float32)).cuda()
    gr = rast.render_backward(res.state, flat)
    torch.cuda.synchronize()
    ref_g = oracle.render_backward(synthetic.widen(g), cams, dL)
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        assert_grad_close(gr[k].cpu().numpy(), ref_g[k], k)
    res.state.release()
