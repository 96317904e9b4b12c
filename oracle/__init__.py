"""AirGS splatting oracle -- TEST INFRASTRUCTURE ONLY.

A plain FP64 CPU restatement of the splatting path of AirGS (arXiv 2512.20943):
decode/apply of streamed updates (Sec. II Eq. 3, Sec. III-B Eq. 5, Sec. III-C),
EWA projection and SH colour of the Gaussian primitive of Sec. II, 16x16 tile
binning with a stable (tile, depth) order, front-to-back blending, the
per-Gaussian blend weight behind usage-frequency pruning (Sec. III-C), the L1
part of Eq. 1, the analytic adjoint, and the clone / split / discard step of
keyframe reconstruction (Sec. III-B).  The arithmetic lives in
``airgs_oracle.cpp``; this module only marshals numpy arrays.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.

Parity pins live in ``tests/test_oracle_*.py``.  The one function without an
external pin is the end-to-end image quality of the paper's trained scenes
(parity unpinned: the paper's dataset is not available).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "airgs_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

# Rasterizer settings used by every definition (3DGS values; see module doc).
DEFAULT_SETTINGS = dict(
    dilation=0.3,
    alpha_max=0.99,
    alpha_min=1.0 / 255.0,
    T_min=1e-4,
    bg=(0.0, 0.0, 0.0),
    tol_px=1e-3,
    tol_rel=1e-5,
    tol_stop=1e-3,
    # relative depth gap under which two list entries may be ordered the other
    # way by the single-precision depth keys (about 2.5 float32 ulps; measured
    # order flips of the GPU's keys came at gaps up to 0.9e-7)
    tol_depth=3e-7,
)

QUAT_COMPOSE = 0
QUAT_ADD = 1


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (plain -O2, single-threaded)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", _LIB_PATH + ".tmp", _SRC]
        subprocess.run(cmd, check=True)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.orc_sh_eval.argtypes = [ctypes.c_int, P, P, P]
        lib.orc_decode_apply.argtypes = [ctypes.c_int64, P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P, P, P, P]
        lib.orc_project.argtypes = [ctypes.c_int64, ctypes.c_int] + [P] * 7 + [P] * 10
        lib.orc_bin_sort.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int64]
        lib.orc_bin_sort.restype = ctypes.c_int64
        lib.orc_render.argtypes = [ctypes.c_int64, ctypes.c_int] + [P] * 5 + [ctypes.c_int, P, P] + [P] * 9
        lib.orc_render_backward.argtypes = [ctypes.c_int64, ctypes.c_int] + [P] * 5 + [ctypes.c_int, P, P] + [P] * 9
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def settings_array(**kw) -> np.ndarray:
    s = dict(DEFAULT_SETTINGS)
    s.update(kw)
    return np.array(
        [s["dilation"], s["alpha_max"], s["alpha_min"], s["T_min"], *s["bg"], s["tol_px"], s["tol_rel"], s["tol_stop"],
         s["tol_depth"]],
        dtype=np.float64,
    )


def camera_array(cam: dict) -> np.ndarray:
    """Flatten a camera dict (width, height, fx, fy, cx, cy, near, viewmat 4x4)."""
    vm = np.asarray(cam["viewmat"], dtype=np.float64).reshape(4, 4)
    return np.concatenate(
        [
            np.array([cam["width"], cam["height"], cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam.get("near", 0.2)],
                     dtype=np.float64),
            vm.reshape(-1),
        ]
    )


def sh_eval(degree: int, direction, with_grad: bool = False):
    """Real SH basis (3DGS sign convention) at a unit direction."""
    lib = _load()
    K = (degree + 1) ** 2
    d = _f64(direction)
    Y = np.zeros(K)
    dY = np.zeros((K, 3)) if with_grad else None
    if lib.orc_sh_eval(degree, _p(d), _p(Y), _p(dY)) != 0:
        raise ValueError("bad degree")
    return (Y, dY) if with_grad else Y


def decode_apply(update_map, lo, hi, base_means, base_quats, quat_mode: int = QUAT_COMPOSE):
    """Decode a [7, H, W] uint16 map and apply it to base means/quats."""
    lib = _load()
    m = np.ascontiguousarray(update_map, dtype=np.uint16)
    assert m.ndim == 3 and m.shape[0] == 7
    bm, bq = _f64(base_means), _f64(base_quats)
    N = bm.shape[0]
    om, oq = np.zeros((N, 3)), np.zeros((N, 4))
    rc = lib.orc_decode_apply(N, _p(m), m.shape[2], m.shape[1], _p(_f64(lo)), _p(_f64(hi)), quat_mode, _p(bm),
                              _p(bq), _p(om), _p(oq))
    if rc != 0:
        raise ValueError("N exceeds the map's pixel count")
    return om, oq


def _params(g):
    return (_f64(g["means"]), _f64(g["log_scales"]), _f64(g["quats"]), _f64(g["opacity_logit"]), _f64(g["sh"]))


def project(g: dict, cam: dict, **settings):
    lib = _load()
    means, ls, qs, ol, sh = _params(g)
    N = means.shape[0]
    deg = int(g["sh_degree"])
    out = dict(
        mean2d=np.zeros((N, 2)), conic=np.zeros((N, 3)), radius=np.zeros(N, np.int32), depth=np.zeros(N),
        rect=np.zeros((N, 4), np.int32), rgb=np.zeros((N, 3)), clamp=np.zeros(N, np.uint8), opacity=np.zeros(N),
        visible=np.zeros(N, np.uint8), ambig=np.zeros(N, np.uint8),
    )
    rc = lib.orc_project(N, deg, _p(means), _p(ls), _p(qs), _p(ol), _p(sh), _p(camera_array(cam)),
                         _p(settings_array(**settings)), _p(out["mean2d"]), _p(out["conic"]), _p(out["radius"]),
                         _p(out["depth"]), _p(out["rect"]), _p(out["rgb"]), _p(out["clamp"]), _p(out["opacity"]),
                         _p(out["visible"]), _p(out["ambig"]))
    if rc != 0:
        raise ValueError("bad sh degree")
    return out


def bin_sort(mean2d, radius, depth, visible, width: int, height: int):
    """Tile lists for given centres, radii, depths (any precision, widened)."""
    lib = _load()
    m2 = _f64(mean2d)
    N = m2.shape[0]
    r = np.ascontiguousarray(radius, dtype=np.int32)
    d = _f64(depth)
    vis = np.ascontiguousarray(visible, dtype=np.uint8)
    ntiles = ((width + 15) // 16) * ((height + 15) // 16)
    ranges = np.zeros((ntiles, 2), np.int64)
    n = lib.orc_bin_sort(N, _p(m2), _p(r), _p(d), _p(vis), width, height, _p(ranges), None, 0)
    lst = np.zeros(max(n, 1), np.int32)
    lib.orc_bin_sort(N, _p(m2), _p(r), _p(d), _p(vis), width, height, _p(ranges), _p(lst), n)
    return ranges, lst[:n]


def _cams(cams):
    return np.ascontiguousarray(np.stack([camera_array(c) for c in cams]), dtype=np.float64)


def _windows(windows, n):
    if windows is None:
        return None
    w = np.ascontiguousarray(np.asarray(windows, np.int32).reshape(n, 4))
    return w


def render(g: dict, cams, windows=None, **settings):
    """Forward over several views.  Returns a dict with per-view lists of
    rgb [3,H,W], T [H,W], n_contrib [H,W], ambig [H,W], and the per-Gaussian
    importance weight/count and ambiguity flags, and the evaluated pair count.
    windows (optional, per view (x0, y0, x1, y1)): blend only those pixels."""
    lib = _load()
    means, ls, qs, ol, sh = _params(g)
    N = means.shape[0]
    sizes = [(int(c["height"]), int(c["width"])) for c in cams]
    tot = sum(h * w for h, w in sizes)
    rgb = np.zeros(3 * tot)
    T = np.zeros(tot)
    nc = np.zeros(tot, np.int32)
    amb = np.zeros(tot, np.uint8)
    w = np.zeros(N)
    cnt = np.zeros(N, np.int64)
    gamb = np.zeros(N, np.uint8)
    pairs = np.zeros(1, np.int64)
    rc = lib.orc_render(N, int(g["sh_degree"]), _p(means), _p(ls), _p(qs), _p(ol), _p(sh), len(cams), _p(_cams(cams)),
                        _p(settings_array(**settings)), _p(rgb), _p(T), _p(nc), _p(w), _p(cnt), _p(amb), _p(gamb),
                        _p(pairs), _p(_windows(windows, len(cams))))
    if rc != 0:
        raise ValueError("bad sh degree")
    out = dict(rgb=[], T=[], n_contrib=[], ambig=[], importance_w=w, importance_cnt=cnt, gauss_ambig=gamb,
               pairs=int(pairs[0]))
    off = 0
    for h, wd in sizes:
        hw = h * wd
        out["rgb"].append(rgb[3 * off:3 * (off + hw)].reshape(3, h, wd))
        out["T"].append(T[off:off + hw].reshape(h, wd))
        out["n_contrib"].append(nc[off:off + hw].reshape(h, wd))
        out["ambig"].append(amb[off:off + hw].reshape(h, wd).astype(bool))
        off += hw
    return out


def render_backward(g: dict, cams, dL_drgb, windows=None, densify=False, **settings):
    """Analytic gradients of sum(dL_drgb * rgb) w.r.t. the raw parameters.
    dL_drgb is a list of [3,H,W] arrays, one per view; with windows, dL_drgb
    must be zero outside them (only window pixels are replayed)."""
    lib = _load()
    means, ls, qs, ol, sh = _params(g)
    N = means.shape[0]
    K = sh.shape[1]
    flat = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).reshape(-1) for x in dL_drgb]))
    gm, gl, gq, go, gs = np.zeros((N, 3)), np.zeros((N, 3)), np.zeros((N, 4)), np.zeros(N), np.zeros((N, K, 3))
    dg, dv = (np.zeros(N), np.zeros(N, np.int64)) if densify else (None, None)
    rc = lib.orc_render_backward(N, int(g["sh_degree"]), _p(means), _p(ls), _p(qs), _p(ol), _p(sh), len(cams),
                                 _p(_cams(cams)), _p(settings_array(**settings)), _p(flat), _p(gm), _p(gl), _p(gq),
                                 _p(go), _p(gs), _p(_windows(windows, len(cams))), _p(dg), _p(dv))
    if rc != 0:
        raise ValueError("bad sh degree")
    out = dict(means=gm, log_scales=gl, quats=gq, opacity_logit=go, sh=gs)
    if densify:
        out["densify_grad"], out["densify_views"] = dg, dv
    return out


def prune_mask(importance, n_prune):
    """Usage-frequency pruning p(.) (Sec. III-C): keep = 0 for the n_prune
    Gaussians of smallest blend weight, equal weights pruning the lower index
    first (a stable ascending sort); negative and NaN weights count as 0."""
    w = np.asarray(importance, np.float64).copy()
    w[~(w > 0)] = 0.0
    order = np.argsort(w, kind="stable")
    keep = np.ones(w.shape[0], np.uint8)
    keep[order[:n_prune]] = 0
    return keep


def prune_delta(D_t, D_sent, keep):
    """d'_t = p(D_t - D'_{t-1}) and D'_t = D'_{t-1} + d'_t (Sec. III-C), channel-major [C, n]."""
    D_t = np.asarray(D_t, np.float64)
    D_sent = np.asarray(D_sent, np.float64)
    d = np.where(np.asarray(keep)[None, :] != 0, D_t - D_sent, 0.0)
    return d, D_sent + d


def apply_delta(base_means, base_quats, delta, quat_add=False):
    """Frame state from a decoded float delta [7, n]: means + (dx, dy, dz) and
    q = normalize(dq (x) q) (Hamilton product) or q + dq."""
    bm = np.asarray(base_means, np.float64)
    bq = np.asarray(base_quats, np.float64)
    d = np.asarray(delta, np.float64)
    means = bm + d[0:3].T
    if quat_add:
        return means, bq + d[3:7].T
    w1, x1, y1, z1 = d[3], d[4], d[5], d[6]
    w2, x2, y2, z2 = bq[:, 0], bq[:, 1], bq[:, 2], bq[:, 3]
    q = np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                  w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                  w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                  w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], axis=1)
    return means, q / np.linalg.norm(q, axis=1, keepdims=True)


def densify_classes(log_scales, opacity_logit, select, size_threshold, min_opacity=0.0):
    """Per-Gaussian decisions of the densification step (see densify_apply):
    (keep, clone, split) boolean arrays.  Both comparisons are taken in float32,
    on the log scale and on the logit (monotone in the scale and the opacity),
    against thresholds rounded once to float32 from float64:
      large  <=>  some log_scale_k > float32(log size_threshold)  (the largest scale above it)
      alive  <=>  not logit < float32(log(m / (1 - m))), m = min_opacity (-inf for m = 0)
    (written so that a NaN component or logit decides as a comparison with NaN does)."""
    ls = np.asarray(log_scales, np.float32).reshape(-1, 3)
    lo = np.asarray(opacity_logit, np.float32).reshape(-1)
    sel = np.asarray(select).reshape(-1) != 0
    ls_thr = np.float32(np.log(np.float64(size_threshold)))
    large = (ls > ls_thr).any(axis=1)
    if min_opacity > 0.0:
        lo_thr = np.float32(np.log(np.float64(min_opacity) / (1.0 - np.float64(min_opacity))))
    else:
        lo_thr = np.float32(-np.inf)
    alive = ~(lo < lo_thr)
    return alive & ~(sel & large), alive & sel & ~large, alive & sel & large


def quat_to_rotation(q):
    """Rotation matrices [n, 3, 3] of quaternions (w, x, y, z) [n, 4], normalised first."""
    q = np.asarray(q, np.float64).reshape(-1, 4)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], axis=1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], axis=1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], axis=1)], axis=1)


def densify_apply(g: dict, select, z, size_threshold, split_factor=1.6, min_opacity=0.0):
    """The clone / split / discard step of keyframe reconstruction (Sec. III-B:
    Gaussians in high-gradient regions are cloned or split, low-opacity ones are
    discarded), with the clone and split rules of the adaptive density control
    of 3D Gaussian Splatting, whose training the paper's keyframe step builds on:
      selected and small (largest scale at most size_threshold): kept, and an
        identical copy added;
      selected and large: replaced by two children that sample the Gaussian as
        a density: mean_j = mean + R(q/|q|) diag(exp(log_scale)) z[i, j],
        log_scale_j = log_scale - log(split_factor) (the scale divided by
        split_factor), quaternion, opacity logit and SH copied;
      opacity below min_opacity: discarded, with its copy or children.
    z [n, 2, 3] are the caller's standard normal samples.  Decisions as in
    densify_classes.  Output (float64): the surviving originals in index order,
    then the copies in index order, then the children (child 0, child 1 of
    each split Gaussian) in index order; parent[j] = input index of output j."""
    means = np.asarray(g["means"], np.float64).reshape(-1, 3)
    n = means.shape[0]
    log_s = np.asarray(g["log_scales"], np.float64).reshape(n, 3)
    quats = np.asarray(g["quats"], np.float64).reshape(n, 4)
    op = np.asarray(g["opacity_logit"], np.float64).reshape(n)
    sh = np.asarray(g["sh"], np.float64).reshape(n, -1)
    keep, clone, split = densify_classes(g["log_scales"], g["opacity_logit"], select, size_threshold, min_opacity)
    ik, ic, isp = np.nonzero(keep)[0], np.nonzero(clone)[0], np.nonzero(split)[0]
    zz = np.asarray(z, np.float64).reshape(n, 2, 3)[isp]                    # [m, 2, 3]
    R = quat_to_rotation(quats[isp])                                          # [m, 3, 3]
    offs = np.einsum("mab,mjb->mja", R, np.exp(log_s[isp])[:, None, :] * zz)  # R (s * z_j)
    child_means = (means[isp][:, None, :] + offs).reshape(-1, 3)
    parent = np.concatenate([ik, ic, np.repeat(isp, 2)])
    out = dict(means=np.concatenate([means[ik], means[ic], child_means]),
               log_scales=np.concatenate([log_s[ik], log_s[ic],
                                          np.repeat(log_s[isp] - np.log(np.float64(split_factor)), 2, axis=0)]),
               quats=quats[parent], opacity_logit=op[parent], sh=sh[parent], parent=parent.astype(np.int64))
    return out


def ssim_window(radius=5, sigma=1.5):
    """Normalised 1D Gaussian weights; the 2D window is their outer product."""
    j = np.arange(-radius, radius + 1, dtype=np.float64)
    w = np.exp(-j * j / (2.0 * sigma * sigma))
    return w / w.sum()


def _blur(img, w):
    """2D zero-padded 'same' convolution of one plane with the window w w^T
    (scipy.signal.convolve2d; the window is symmetric)."""
    from scipy.signal import convolve2d
    return convolve2d(img, np.outer(w, w), mode="same", boundary="fill", fillvalue=0.0)


def ssim_map(x, y, C1=0.01 ** 2, C2=0.03 ** 2):
    """Per-pixel SSIM of two planes (the map l3dgs_loss_grad averages)."""
    w = ssim_window()
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = _blur(x, w), _blur(y, w)
    mxx, myy, mxy = _blur(x * x, w), _blur(y * y, w), _blur(x * y, w)
    return ((2 * mx * my + C1) * (2 * (mxy - mx * my) + C2) /
            ((mx * mx + my * my + C1) * ((mxx - mx * mx) + (myy - my * my) + C2)))


def l3dgs_loss_grad(rgb_views, target_views, lam=0.2, C1=0.01 ** 2, C2=0.03 ** 2):
    """L_3DGS of Eq. 1: L = (1 - lam) L1 + lam (1 - SSIM), SSIM with an 11x11
    Gaussian window (sigma 1.5), zero padding, averaged over views, channels and
    pixels; returns (L, L1, SSIM, [dL/d rgb per view]).  The gradient is the
    window correlation of the SSIM map's partials with respect to the local
    moments mu_x, E[x^2], E[xy]."""
    w = ssim_window()
    total = sum(np.asarray(r).size for r in rgb_views)
    s_sum, l1_sum, grads = 0.0, 0.0, []
    for rv, tv in zip(rgb_views, target_views):
        rv = np.asarray(rv, np.float64)
        tv = np.asarray(tv, np.float64)
        g = np.zeros_like(rv)
        for c in range(rv.shape[0]):
            x, y = rv[c], tv[c]
            mx, my = _blur(x, w), _blur(y, w)
            mxx, myy, mxy = _blur(x * x, w), _blur(y * y, w), _blur(x * y, w)
            A = 2 * mx * my + C1
            B = 2 * (mxy - mx * my) + C2
            Cc = mx * mx + my * my + C1
            D = (mxx - mx * mx) + (myy - my * my) + C2
            S = A * B / (Cc * D)
            s_sum += S.sum()
            P1 = 2 * my * (B - A) / (Cc * D) - 2 * mx * S / Cc + 2 * mx * S / D
            P2 = -S / D
            P3 = 2 * A / (Cc * D)
            dS = _blur(P1, w) + 2 * x * _blur(P2, w) + y * _blur(P3, w)
            d = x - y
            l1_sum += np.abs(d).sum()
            g[c] = -lam * dS / total + (1 - lam) * np.sign(d) / total
        grads.append(g)
    ssim, l1 = s_sum / total, l1_sum / total
    return (1 - lam) * l1 + lam * (1 - ssim), l1, ssim, grads


def l1_loss_grad(rgb_views, target_views):
    """L1 part of Eq. 1: mean |C - target| over views, pixels and channels, and
    its gradient sign(C - target) / (3 sum_v H_v W_v), sign(0) = 0."""
    n = sum(np.asarray(r).size for r in rgb_views)
    loss = sum(np.abs(np.asarray(r, np.float64) - np.asarray(t, np.float64)).sum()
               for r, t in zip(rgb_views, target_views)) / n
    grads = [np.sign(np.asarray(r, np.float64) - np.asarray(t, np.float64)) / n for r, t in zip(rgb_views, target_views)]
    return loss, grads
