"""Seeded synthetic inputs shaped like the AirGS workloads.

This module only draws random numbers and builds cameras; it holds none of the
rendering arithmetic.  Both the CUDA path's tests/benchmark and the oracle take
their inputs from here.  The real workloads (the HiFi4G captures, 81 views at
3840x2160, 30 fps) are not available; these scenes stand in for them with the
Gaussian counts, SH degree, resolutions and update-map sizes of each workload.

All arrays are float32 (the precision the CUDA path consumes); tests widen the
same float32 values to float64 before handing them to the oracle.
"""
from __future__ import annotations

import math

import numpy as np

UPDATE_CHANNELS = 7  # dx, dy, dz, qw, qx, qy, qz


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def gaussians(n, seed, *, mean_mode="normal", mean_scale=(3.0, 2.0, 3.0), log_scale=(-4.0, 0.7), sh_degree=3,
              sh_std=0.2, opacity_std=1.0, rgb_dc=False):
    """Random Gaussians.

    mean_mode 'uniform': means ~ U[-1, 1]^3 * mean_scale; 'normal': N(0, 1) * mean_scale.
    log-scales ~ N(log_scale[0], log_scale[1]); quaternions uniform on S^3;
    opacity logits ~ N(0, opacity_std).  SH coefficients ~ N(0, sh_std), or,
    with rgb_dc, degree-0 coefficients drawn so that the rendered colour is
    U[0, 1]: dc = (u - 0.5) * 2 sqrt(pi), since the degree-0 basis function is
    the constant 1 / (2 sqrt(pi)) and 0.5 is added to the colour.
    """
    rng = np.random.default_rng(seed)
    ms = np.asarray(mean_scale, dtype=np.float64)
    if mean_mode == "uniform":
        means = rng.uniform(-1.0, 1.0, (n, 3)) * ms
    else:
        means = rng.standard_normal((n, 3)) * ms
    log_scales = rng.normal(log_scale[0], log_scale[1], (n, 3))
    quats = _unit_quats(rng, n)
    opacity_logit = rng.normal(0.0, opacity_std, n)
    K = (sh_degree + 1) ** 2
    if rgb_dc:
        u = rng.uniform(0.0, 1.0, (n, 1, 3))
        sh = (u - 0.5) * (2.0 * math.sqrt(math.pi))
        if K > 1:
            sh = np.concatenate([sh, np.zeros((n, K - 1, 3))], axis=1)
    else:
        sh = rng.normal(0.0, sh_std, (n, K, 3))
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return dict(sh_degree=sh_degree, means=f(means), log_scales=f(log_scales), quats=f(quats),
                opacity_logit=f(opacity_logit), sh=f(sh))


def look_at(position, target=(0.0, 0.0, 0.0), down=(0.0, 1.0, 0.0)):
    """World->camera 4x4 (row-major) for a camera at `position` looking at
    `target`; camera axes x right, y down, z forward."""
    p = np.asarray(position, np.float64)
    z = np.asarray(target, np.float64) - p
    z /= np.linalg.norm(z)
    d = np.asarray(down, np.float64)
    y = d - np.dot(d, z) * z
    if np.linalg.norm(y) < 1e-9:
        y = np.array([0.0, 0.0, 1.0]) - z[2] * z
    y /= np.linalg.norm(y)
    x = np.cross(y, z)
    R = np.stack([x, y, z])
    vm = np.eye(4)
    vm[:3, :3] = R
    vm[:3, 3] = -R @ p
    return vm


def camera(position, width, height, fov_x_deg=None, fx=None, near=0.2, target=(0.0, 0.0, 0.0)):
    if fx is None:
        fx = width / (2.0 * math.tan(math.radians(fov_x_deg) / 2.0))
    return dict(width=int(width), height=int(height), fx=float(fx), fy=float(fx), cx=width / 2.0, cy=height / 2.0,
                near=float(near), viewmat=look_at(position, target))


def arc_cameras(n, radius=10.0, arc_deg=120.0, width=1352, height=1014, fov_x_deg=60.0):
    """n cameras evenly spaced on a horizontal arc (height 0) looking at the origin."""
    out = []
    for k in range(n):
        th = math.radians(-arc_deg / 2.0 + arc_deg * (k / (n - 1) if n > 1 else 0.5))
        pos = (radius * math.sin(th), 0.0, -radius * math.cos(th))
        out.append(camera(pos, width, height, fov_x_deg=fov_x_deg))
    return out


def sphere_pose(rng, radius=3.0):
    v = rng.standard_normal(3)
    v /= np.linalg.norm(v)
    return v * radius


def update_map(n_gauss, seed, size=768, pos_std=0.01, pos_range=0.08, rot_std=0.01, w_range=(0.99, 1.0),
               xyz_range=0.08):
    """One frame's 7-channel 16-bit update map (one Gaussian per pixel,
    row-major, one attribute per channel).  Returns (map[7, size, size] uint16,
    lo[7], hi[7]); the value of channel c is lo[c] + u (hi[c] - lo[c]) / 65535.
    Position offsets ~ N(0, pos_std); the rotation delta is normalize(1, eps),
    eps ~ N(0, rot_std)^3.  Pixels past n_gauss hold a zero offset and the
    identity rotation."""
    rng = np.random.default_rng(seed)
    P = size * size
    if n_gauss > P:
        raise ValueError("more Gaussians than map pixels")
    lo = np.array([-pos_range] * 3 + [w_range[0]] + [-xyz_range] * 3, np.float32)
    hi = np.array([pos_range] * 3 + [w_range[1]] + [xyz_range] * 3, np.float32)
    vals = np.zeros((UPDATE_CHANNELS, P))
    vals[3] = 1.0
    vals[0:3, :n_gauss] = rng.normal(0.0, pos_std, (3, n_gauss))
    dq = np.concatenate([np.ones((1, n_gauss)), rng.normal(0.0, rot_std, (3, n_gauss))], axis=0)
    dq /= np.linalg.norm(dq, axis=0, keepdims=True)
    vals[3:7, :n_gauss] = dq
    lo64, hi64 = lo.astype(np.float64)[:, None], hi.astype(np.float64)[:, None]
    u = np.rint((vals - lo64) / (hi64 - lo64) * 65535.0)
    u = np.clip(u, 0, 65535).astype(np.uint16)
    return u.reshape(UPDATE_CHANNELS, size, size), lo, hi


def target_images(cams, seed):
    rng = np.random.default_rng(seed)
    return [rng.uniform(0.0, 1.0, (3, c["height"], c["width"])).astype(np.float32) for c in cams]


# ---------------------------------------------------------------- workloads
def plain_forward_scene():
    """Plain forward render: 2,000 Gaussians, means U[-1,1]^3, log-scales
    N(-3, 0.5), opacity sigmoid(N(0,1)), SH degree 0 with RGB U[0,1]; one
    128x128 pinhole camera at z=-4 looking at the origin, fx=fy=128; seed 0."""
    g = gaussians(2000, 0, mean_mode="uniform", mean_scale=(1.0, 1.0, 1.0), log_scale=(-3.0, 0.5), sh_degree=0,
                  rgb_dc=True)
    cam = camera((0.0, 0.0, -4.0), 128, 128, fx=128.0)
    return g, [cam]


def per_frame_training_scene(n=200_000, n_views=20, width=1352, height=1014, seed=0):
    """Per-frame training step: 200k Gaussians, means N(0,1)*(3,2,3), log-scales
    N(-4, 0.7), SH degree 3 ~ N(0, 0.2); 20 cameras on a 120-degree arc at
    1352x1014 (60-degree horizontal FOV, radius 10); targets U[0,1] (seed 1)."""
    g = gaussians(n, seed)
    cams = arc_cameras(n_views, width=width, height=height)
    return g, cams


def streaming_scene(n=300_000, seed=0):
    """Batched streaming training: a 300k-Gaussian anchor drawn like the
    per-frame training scene; frame t's update map comes from update_map(n,
    1000 + t); views 8t mod 20 ... of the 20-camera arc at 1352x1014."""
    g = gaussians(n, seed)
    cams = arc_cameras(20)
    return g, cams


def streaming_views(cams, frame, per_launch=8):
    return [cams[(per_launch * frame + k) % len(cams)] for k in range(per_launch)]


def serving_scene(n=500_000, seed=0):
    """Serving: 500k anchor, means N(0, 0.7^2 I), log-scales N(-4.5, 0.7), SH3 N(0, 0.2)."""
    return gaussians(n, seed, mean_scale=(0.7, 0.7, 0.7), log_scale=(-4.5, 0.7))


SERVING_SIZES = ((640, 480), (1280, 720), (1920, 1080))


def serving_requests(n_viewers=64, rate_hz=30.0, duration_s=10.0, seed=4, radius=3.0, fov_x_deg=60.0):
    """Open-loop Poisson render requests: each of n_viewers issues requests at
    rate_hz; resolution uniform over SERVING_SIZES; pose uniform on a sphere of
    `radius` looking at the origin.  Returns a time-sorted list of
    (arrival_s, viewer, camera)."""
    rng = np.random.default_rng(seed)
    reqs = []
    for v in range(n_viewers):
        t = 0.0
        while True:
            t += rng.exponential(1.0 / rate_hz)
            if t >= duration_s:
                break
            w, h = SERVING_SIZES[rng.integers(len(SERVING_SIZES))]
            reqs.append((t, v, camera(sphere_pose(rng, radius), w, h, fov_x_deg=fov_x_deg)))
    reqs.sort(key=lambda r: r[0])
    return reqs


def large_scene(n=2_000_000, n_views=16, seed=0):
    """Large scene: 2M Gaussians SH3, log-scales N(-5, 0.8), opacity logits
    N(0, 1.5), means like the per-frame scene; 16 views at 3840x2160 on the arc."""
    g = gaussians(n, seed, log_scale=(-5.0, 0.8), opacity_std=1.5)
    cams = arc_cameras(n_views, width=3840, height=2160)
    return g, cams


def widen(g):
    """The same float32 parameters as float64 arrays (for the oracle)."""
    out = dict(g)
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        out[k] = np.asarray(g[k], dtype=np.float64)
    return out
