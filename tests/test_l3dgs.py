"""The L_3DGS loss of Eq. 1 (L1 + D-SSIM, lambda = 0.2): the oracle against
SSIM's defining properties, a direct per-window computation and central
differences; the CUDA kernels against the oracle."""
import numpy as np
import pytest

import oracle


def _ssim_direct(x, y, C1=1e-4, C2=9e-4):
    """SSIM map by explicit 11x11 windows (zero outside the image)."""
    w1 = oracle.ssim_window()
    W2 = np.outer(w1, w1)
    H, Wd = x.shape
    xp = np.pad(x, 5)
    yp = np.pad(y, 5)
    out = np.zeros_like(x)
    for r in range(H):
        for c in range(Wd):
            a = xp[r:r + 11, c:c + 11]
            b = yp[r:r + 11, c:c + 11]
            mx, my = (W2 * a).sum(), (W2 * b).sum()
            vx, vy = (W2 * a * a).sum() - mx * mx, (W2 * b * b).sum() - my * my
            cxy = (W2 * a * b).sum() - mx * my
            out[r, c] = (2 * mx * my + C1) * (2 * cxy + C2) / ((mx * mx + my * my + C1) * (vx + vy + C2))
    return out


def test_ssim_identity_symmetry_and_direct_windows():
    rng = np.random.default_rng(0)
    x = rng.random((3, 19, 23))
    y = np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1)
    L, l1, ssim, _ = oracle.l3dgs_loss_grad([x], [x])
    assert abs(ssim - 1.0) < 1e-12 and l1 == 0.0 and abs(L) < 1e-12
    _, _, s_xy, _ = oracle.l3dgs_loss_grad([x], [y])
    _, _, s_yx, _ = oracle.l3dgs_loss_grad([y], [x])
    assert abs(s_xy - s_yx) < 1e-12 and s_xy < 1.0
    direct = np.mean([_ssim_direct(x[c], y[c]) for c in range(3)])
    assert abs(direct - s_xy) < 1e-12
    assert oracle.ssim_window().sum() == pytest.approx(1.0, abs=1e-15)


def test_ssim_closed_forms_away_from_the_border():
    """Where the 11x11 window lies inside the image: constant planes a and b
    give the luminance term (2ab + C1) / (a^2 + b^2 + C1) alone (no variance);
    y = x + c (same variance, covariance = variance) gives the same luminance
    term of the local means; y = s x gives the contrast-structure term
    (2 s v + C2) / ((1 + s^2) v + C2) (v the local variance) times the
    luminance term of the local means."""
    C1, C2 = 1e-4, 9e-4
    a, b = 0.3, 0.7
    S = oracle.ssim_map(np.full((20, 24), a), np.full((20, 24), b))
    assert np.allclose(S[5:-5, 5:-5], (2 * a * b + C1) / (a * a + b * b + C1), rtol=0, atol=1e-14)
    rng = np.random.default_rng(3)
    x = rng.random((30, 31))
    w = oracle.ssim_window()
    W2 = np.outer(w, w)
    for r, c in ((12, 9), (5, 5), (24, 25)):
        win = x[r - 5:r + 6, c - 5:c + 6]
        mu, var = (W2 * win).sum(), (W2 * win * win).sum() - (W2 * win).sum() ** 2
        cshift = 0.2
        S_shift = oracle.ssim_map(x, x + cshift)[r, c]
        lum = (2 * mu * (mu + cshift) + C1) / (mu ** 2 + (mu + cshift) ** 2 + C1)
        assert abs(S_shift - lum) < 1e-12
        s = 0.6
        S_scale = oracle.ssim_map(x, s * x)[r, c]
        lum_s = (2 * mu * s * mu + C1) / (mu ** 2 + (s * mu) ** 2 + C1)
        cs = (2 * s * var + C2) / ((1 + s * s) * var + C2)
        assert abs(S_scale - lum_s * cs) < 1e-12


def test_l3dgs_gradient_central_differences():
    rng = np.random.default_rng(1)
    x = rng.random((3, 9, 12))
    y = rng.random((3, 9, 12))
    L0, _, _, (g,) = oracle.l3dgs_loss_grad([x], [y], lam=0.2)
    h = 1e-6
    for _ in range(60):
        c, r, k = rng.integers(3), rng.integers(9), rng.integers(12)
        if abs(x[c, r, k] - y[c, r, k]) < 1e-3:
            continue  # keep away from the L1 kink
        xp, xm = x.copy(), x.copy()
        xp[c, r, k] += h
        xm[c, r, k] -= h
        fd = (oracle.l3dgs_loss_grad([xp], [y])[0] - oracle.l3dgs_loss_grad([xm], [y])[0]) / (2 * h)
        assert abs(fd - g[c, r, k]) < 1e-7 * max(1.0, abs(fd)), (c, r, k)


@pytest.mark.gpu
def test_l3dgs_kernels_match_oracle():
    import torch
    import synthetic
    from paper_2512_20943_b300 import Rasterizer
    cams = [synthetic.camera((0, 0, -4.0), 100, 70, fx=80.0), synthetic.camera((0, 0, -4.0), 33, 17, fx=30.0),
            synthetic.camera((0, 0, -4.0), 256, 200, fx=220.0)]
    rng = np.random.default_rng(2)
    xs = [rng.random((3, c["height"], c["width"])).astype(np.float32) for c in cams]
    ys = [np.clip(x + rng.normal(0, 0.2, x.shape), 0, 1).astype(np.float32) for x in xs]
    rast = Rasterizer()
    flat = lambda a: torch.from_numpy(np.concatenate([v.reshape(-1) for v in a])).cuda()
    loss, grad = rast.l3dgs_loss(cams, flat(xs), flat(ys), 0.2)
    torch.cuda.synchronize()
    L, l1, ssim, g_ref = oracle.l3dgs_loss_grad(xs, ys, 0.2)
    lo = loss.cpu().numpy()
    assert abs(lo[0] - L) < 1e-5 and abs(lo[1] - l1) < 1e-6 and abs(lo[2] - ssim) < 1e-5
    g = grad.cpu().numpy()
    ref = np.concatenate([v.reshape(-1) for v in g_ref])
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert rel < 1e-4, rel


@pytest.mark.gpu
def test_l3dgs_kernels_match_oracle_full_size_view():
    """A full 1352x1014 view (the training views' size: 43 x 32 output tiles of
    the fused tile kernel, ragged in both directions) and a 333x217 view in one
    call: loss terms and the gradient against the oracle (relative L2 1e-4 and
    1e-3 of the largest magnitude elementwise).  Inputs are smooth fields plus
    noise, so that the SSIM map varies across the window scales."""
    import torch
    import synthetic
    from paper_2512_20943_b300 import Rasterizer
    cams = [synthetic.camera((0, 0, -4.0), 1352, 1014, fx=1170.0), synthetic.camera((0, 0, -4.0), 333, 217, fx=300.0)]
    rng = np.random.default_rng(12)
    xs, ys = [], []
    for c in cams:
        h, w = c["height"], c["width"]
        yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
        base = np.stack([0.5 + 0.4 * np.sin(xx / (7.0 + 5 * k) + yy / (11.0 + 3 * k)) for k in range(3)])
        x = np.clip(base + rng.normal(0, 0.05, base.shape), 0, 1).astype(np.float32)
        xs.append(x)
        ys.append(np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1).astype(np.float32))
    rast = Rasterizer()
    flat = lambda a: torch.from_numpy(np.concatenate([v.reshape(-1) for v in a])).cuda()
    loss, grad = rast.l3dgs_loss(cams, flat(xs), flat(ys), 0.2)
    torch.cuda.synchronize()
    L, l1, ssim, g_ref = oracle.l3dgs_loss_grad(xs, ys, 0.2)
    lo = loss.cpu().numpy()
    assert abs(lo[0] - L) < 1e-5 and abs(lo[1] - l1) < 1e-6 and abs(lo[2] - ssim) < 1e-5, (lo, L, l1, ssim)
    g = grad.cpu().numpy()
    ref = np.concatenate([v.reshape(-1) for v in g_ref])
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert rel < 1e-4, rel
    assert np.abs(g - ref).max() <= 1e-3 * np.abs(ref).max()
