"""Parity of the device densification step (clone / split / discard of keyframe
reconstruction, Sec. III-B) with the oracle, through the C ABI.

Bars: the output count, the parent map and every copied value (kept
originals, copies, the children's quaternion, opacity and SH) bit-exact; the
children's means within 2e-6 (1 + |value|) and log scales within 1e-6 of the
oracle's float64 values (single-precision rotation, exp and subtraction);
the decisions are float32 comparisons on both sides, so they agree exactly.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synthetic
from tests._helpers import params, to_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rast():
    from paper_2512_20943_b300 import Rasterizer
    return Rasterizer()


def _case(n, deg, seed, sel_frac=0.3):
    """Gaussians whose scales straddle the size threshold 0.05 and whose
    opacities straddle the floor 0.1, unnormalised quaternions, a random
    selection and standard normal samples."""
    g = synthetic.gaussians(n, seed, log_scale=(np.log(0.05), 0.8), sh_degree=deg, opacity_std=2.0)
    rng = np.random.default_rng(seed + 1)
    g["quats"] = np.ascontiguousarray(g["quats"] * rng.uniform(0.5, 2.0, (n, 1)), np.float32)
    sel = (rng.uniform(size=n) < sel_frac).astype(np.uint8)
    z = rng.standard_normal((n, 2, 3)).astype(np.float32)
    return g, sel, z


def _check(out, g, sel, z, size_threshold, split_factor, min_opacity):
    ref = oracle.densify_apply(g, sel, z, size_threshold, split_factor, min_opacity)
    m = ref["parent"].shape[0]
    got = {k: v.cpu().numpy() for k, v in out.items()}
    assert got["parent"].shape[0] == m
    assert np.array_equal(got["parent"].astype(np.int64), ref["parent"])
    K3 = g["sh"].shape[1] * 3
    keep, clone, split = oracle.densify_classes(g["log_scales"], g["opacity_logit"], sel, size_threshold, min_opacity)
    n_copy = int(keep.sum() + clone.sum())
    par = ref["parent"]
    # originals and copies: the input rows, bit for bit
    for k in ("means", "log_scales", "quats", "opacity_logit"):
        assert np.array_equal(got[k][:n_copy], g[k][par[:n_copy]]), k
    assert np.array_equal(got["sh"].reshape(m, K3)[:n_copy], g["sh"].reshape(-1, K3)[par[:n_copy]])
    # children: rotation, opacity and SH copied; means and scales as the oracle's
    assert np.array_equal(got["quats"][n_copy:], g["quats"][par[n_copy:]])
    assert np.array_equal(got["opacity_logit"][n_copy:], g["opacity_logit"][par[n_copy:]])
    assert np.array_equal(got["sh"].reshape(m, K3)[n_copy:], g["sh"].reshape(-1, K3)[par[n_copy:]])
    cm, rm = got["means"][n_copy:].astype(np.float64), ref["means"][n_copy:]
    assert np.all(np.abs(cm - rm) <= 2e-6 * (1.0 + np.abs(rm))), np.abs(cm - rm).max()
    assert np.abs(got["log_scales"][n_copy:] - ref["log_scales"][n_copy:]).max(initial=0.0) <= 1e-6
    return ref, (int(keep.sum()), int(clone.sum()), int(split.sum()))


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
@pytest.mark.parametrize("n", [1, 1023, 1024, 5003])
def test_densify_apply_matches_oracle(rast, n, deg):
    g, sel, z = _case(n, deg, seed=100 + n + deg)
    t = to_cuda(g)
    out = rast.densify_apply(*params(t), torch.from_numpy(sel).cuda(), torch.from_numpy(z).cuda(), 0.05, 1.6, 0.1)
    _check(out, g, sel, z, 0.05, 1.6, 0.1)


def test_densify_apply_every_class_at_size(rast):
    # 70k Gaussians (136 tiles of 512 and a ragged last one): all three classes
    # and discards occur, in every tile
    g, sel, z = _case(70_001, 3, seed=7, sel_frac=0.5)
    t = to_cuda(g)
    out = rast.densify_apply(*params(t), torch.from_numpy(sel).cuda(), torch.from_numpy(z).cuda(), 0.05, 2.0, 0.2)
    _, (k, c, s) = _check(out, g, sel, z, 0.05, 2.0, 0.2)
    assert k > 0 and c > 0 and s > 0 and k + c + 2 * s < 2 * 70_001


def test_densify_apply_unaligned_sh_takes_the_scalar_copy(rast):
    g, sel, z = _case(3001, 3, seed=9)
    t = to_cuda(g)
    flat = torch.empty(t["sh"].numel() + 1, device="cuda")
    sh = flat[1:].view(t["sh"].shape)  # 4 bytes past a 16-byte boundary
    sh.copy_(t["sh"])
    out = rast.densify_apply(t["means"], t["log_scales"], t["quats"], t["opacity_logit"], sh,
                             torch.from_numpy(sel).cuda(), torch.from_numpy(z).cuda(), 0.05, 1.6, 0.1)
    _check(out, g, sel, z, 0.05, 1.6, 0.1)


def test_densify_apply_degenerate_inputs(rast):
    # nothing selected and no floor: the identity; everything below the floor:
    # nothing; no Gaussians: nothing
    g, _, z = _case(2000, 1, seed=3)
    t = to_cuda(g)
    zc = torch.from_numpy(z).cuda()
    none = torch.zeros(2000, dtype=torch.uint8, device="cuda")
    out = rast.densify_apply(*params(t), none, zc, 0.05)
    assert torch.equal(out["parent"].cpu(), torch.arange(2000, dtype=torch.int32))
    assert torch.equal(out["sh"], t["sh"]) and torch.equal(out["means"], t["means"])
    out = rast.densify_apply(*params(t), torch.ones_like(none), zc, 0.05, 1.6, 0.999999)
    assert out["parent"].numel() == 0
    e = {k: v[:0] for k, v in t.items()}
    out = rast.densify_apply(*params(e), none[:0], zc[:0], 0.05)
    assert out["means"].shape == (0, 3)


def test_densify_apply_argument_errors(rast):
    from paper_2512_20943_b300 import AirGSError
    from paper_2512_20943_b300._abi import AIRGS_E_ARG, AIRGS_E_CAPACITY, airgs_densify_out, airgs_gaussians
    g, sel, z = _case(100, 0, seed=5)
    t = to_cuda(g)
    s, zc = torch.from_numpy(sel).cuda(), torch.from_numpy(z).cuda()
    for bad in (dict(size_threshold=0.0), dict(size_threshold=float("nan")), dict(split_factor=-1.0),
                dict(min_opacity=1.0), dict(min_opacity=-0.1)):
        kw = dict(size_threshold=0.05, split_factor=1.6, min_opacity=0.0)
        kw.update(bad)
        with pytest.raises(AirGSError) as ei:
            rast.densify_apply(*params(t), s, zc, **kw)
        assert ei.value.code == AIRGS_E_ARG
    # a capacity below 2 n is refused before any launch
    bufs = [torch.empty(199 * c, device="cuda") for c in (3, 3, 4, 1, 3)]
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    gs = airgs_gaussians(100, 0, *(t[k].data_ptr() for k in ("means", "log_scales", "quats", "opacity_logit", "sh")))
    d = airgs_densify_out(199, *(b.data_ptr() for b in bufs), None, n_out.data_ptr())
    rc = rast.lib.airgs_densify_apply(rast.ctx, ctypes.byref(gs), s.data_ptr(), zc.data_ptr(), 0.05, 1.6, 0.0,
                                      ctypes.byref(d))
    assert rc == AIRGS_E_CAPACITY


def test_densify_select_then_apply_full_size(rast):
    # the streaming anchor's size (300k SH3) with its densification statistics
    # from one training backward over 8 views: select, split or clone, compare
    n = 300_000
    g = synthetic.gaussians(n, 21, sh_degree=3)
    t = to_cuda(g)
    rng = np.random.default_rng(22)
    cams = [synthetic.camera(synthetic.sphere_pose(rng, 6.0), 1352, 1014, fov_x_deg=60.0) for _ in range(8)]
    res = rast.render_gaussians(*params(t), cams, save=True)
    target = torch.rand_like(res.rgb)
    dg = torch.zeros(n, device="cuda")
    dv = torch.zeros(n, dtype=torch.int32, device="cuda")
    rast.render_backward_ex(res.state, target=target, densify=(dg, dv))
    vis = dv > 0
    thr_g = float(torch.quantile((dg[vis] / dv[vis].float()).double(), 0.7))  # about 30 % of the visible ones
    sel = rast.densify_select(dg, dv, thr_g)
    z = torch.randn(n, 2, 3, generator=torch.Generator(device="cuda").manual_seed(23), device="cuda")
    thr = float(np.exp(np.median(g["log_scales"].max(axis=1))))
    out = rast.densify_apply(*params(t), sel, z, thr, 1.6, 0.005)
    sel_np = sel.cpu().numpy()
    assert 0.01 * n < sel_np.sum() < 0.9 * n
    _check(out, g, sel_np, z.cpu().numpy(), thr, 1.6, 0.005)
