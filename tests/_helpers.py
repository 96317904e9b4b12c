"""Shared helpers of the GPU parity tests (inputs and comparisons; no arithmetic
of the method)."""
import numpy as np
import torch

import synthetic

RGB_ATOL = 1e-3        # RGB in [0, 1]: absolute tolerance
GRAD_RTOL = 1e-3       # gradients: ||g - g_ref|| / ||g_ref|| per tensor
GRAD_ELEM = 1e-3       # gradients: |g - g_ref| <= GRAD_ELEM * max |g_ref| elementwise


def to_cuda(g):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in g.items() if k != "sh_degree"}


def params(t):
    return t["means"], t["log_scales"], t["quats"], t["opacity_logit"], t["sh"]


def views_np(flat, cams, channels=3):
    out, off = [], 0
    a = flat.detach().cpu().numpy()
    for c in cams:
        n = channels * c["height"] * c["width"]
        shape = (channels, c["height"], c["width"]) if channels > 1 else (c["height"], c["width"])
        out.append(a[off:off + n].reshape(shape))
        off += n
    return out


def assert_grad_close(g, ref, name):
    g = np.asarray(g, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    nref = np.linalg.norm(ref)
    if nref == 0:
        assert np.abs(g).max() == 0, name
        return
    rel = np.linalg.norm(g - ref) / nref
    elem = np.abs(g - ref).max() / np.abs(ref).max()
    assert rel <= GRAD_RTOL, f"{name}: relative L2 error {rel:.3e}"
    assert elem <= GRAD_ELEM, f"{name}: elementwise error {elem:.3e} of max"


def small_sh3_scene(n=400, seed=21):
    g = synthetic.gaussians(n, seed, mean_mode="uniform", mean_scale=(1.2, 1.0, 1.2), log_scale=(-3.2, 0.5),
                            sh_degree=3, sh_std=0.2)
    cams = [synthetic.camera((0.3, -0.2, -4.0), 100, 70, fov_x_deg=50.0),
            synthetic.camera((2.5, 0.5, -3.0), 64, 48, fov_x_deg=60.0),
            synthetic.camera((-1.0, 0.0, -3.5), 33, 17, fov_x_deg=45.0)]
    return g, cams
