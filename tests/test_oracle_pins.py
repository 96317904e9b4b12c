"""Pins of the FP64 oracle against facts fixed outside it: closed forms of the
pinhole EWA projection, a library spherical-harmonic routine, the telescoping
identity of front-to-back blending, permutation invariance, a brute-force
per-pixel renderer, the threshold rules, quaternion algebra, and central finite
differences of the oracle's own forward for its adjoint."""
import math

import numpy as np
import pytest
import scipy.special as sps

import oracle
import synthetic

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


# ---------------------------------------------------------------- helpers
def one_gaussian(mean, log_scale, quat, logit, rgb, sh_degree=0):
    K = (sh_degree + 1) ** 2
    sh = np.zeros((1, K, 3))
    sh[0, 0] = (np.asarray(rgb, np.float64) - 0.5) * 2.0 * math.sqrt(math.pi)
    return dict(sh_degree=sh_degree, means=np.array([mean], np.float64), log_scales=np.array([log_scale], np.float64),
                quats=np.array([quat], np.float64), opacity_logit=np.array([logit], np.float64), sh=sh)


def concat(gs):
    out = dict(sh_degree=gs[0]["sh_degree"])
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        out[k] = np.concatenate([g[k] for g in gs], axis=0)
    return out


def axis_camera(W=64, H=64, f=64.0, dist=4.0):
    vm = np.eye(4)
    vm[2, 3] = dist  # camera at (0, 0, -dist) looking down +z
    return dict(width=W, height=H, fx=f, fy=f, cx=W / 2.0, cy=H / 2.0, near=0.2, viewmat=vm)


def logit(p):
    return math.log(p / (1 - p))


# ---------------------------------------------------------------- spherical harmonics
def test_sh_matches_library_complex_harmonics():
    """Real basis with the Condon-Shortley phase kept:
    Y_l,m = sqrt2 Re Y_l^m (m > 0), sqrt2 Im Y_l^|m| (m < 0), Y_l^0 (m = 0),
    with Y_l^m from scipy.special.sph_harm_y."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        Y = oracle.sh_eval(3, d)
        for l in range(4):
            for m in range(-l, l + 1):
                c = sps.sph_harm_y(l, abs(m), theta, phi)
                ref = c.real if m == 0 else math.sqrt(2) * (c.real if m > 0 else c.imag)
                assert abs(Y[l * l + l + m] - ref) < 1e-12, (l, m)


def test_sh_orthonormal_by_quadrature():
    """Gauss-Legendre in cos(theta) x uniform phi integrates degree <= 6
    products exactly."""
    x, w = np.polynomial.legendre.leggauss(12)
    phis = np.arange(24) * (2 * math.pi / 24)
    G = np.zeros((16, 16))
    for xi, wi in zip(x, w):
        s = math.sqrt(1 - xi * xi)
        for ph in phis:
            Y = oracle.sh_eval(3, [s * math.cos(ph), s * math.sin(ph), xi])
            G += wi * (2 * math.pi / 24) * np.outer(Y, Y)
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_low_order_closed_forms():
    d = np.array([0.3, -0.5, 0.8])
    d /= np.linalg.norm(d)
    Y = oracle.sh_eval(1, d)
    c0, c1 = 1 / (2 * math.sqrt(math.pi)), math.sqrt(3 / (4 * math.pi))
    assert abs(Y[0] - c0) < 1e-15
    # degree 1 is (-y, z, -x) up to the normalisation
    assert np.allclose(Y[1:], c1 * np.array([-d[1], d[2], -d[0]]), atol=1e-15)


def test_sh_gradient_by_finite_differences():
    rng = np.random.default_rng(5)
    for _ in range(5):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        _, dY = oracle.sh_eval(3, d, with_grad=True)
        # tangential directional derivatives along the sphere
        for _k in range(3):
            t = rng.standard_normal(3)
            t -= t.dot(d) * d
            t /= np.linalg.norm(t)
            h = 1e-5
            yp = oracle.sh_eval(3, (d + h * t) / np.linalg.norm(d + h * t))
            ym = oracle.sh_eval(3, (d - h * t) / np.linalg.norm(d - h * t))
            fd = (yp - ym) / (2 * h)
            assert np.abs(dY @ t - fd).max() < 1e-8


# ---------------------------------------------------------------- projection closed forms
@pytest.mark.parametrize("s,f,d", [(0.05, 64.0, 4.0), (0.2, 100.0, 3.0), (0.01, 1171.0, 10.0)])
def test_centred_isotropic_projection(s, f, d):
    cam = axis_camera(W=128, H=96, f=f, dist=d)
    g = one_gaussian([0, 0, 0], [math.log(s)] * 3, [1, 0, 0, 0], 0.0, [0.5, 0.5, 0.5])
    p = oracle.project(g, cam)
    sig2 = (f * s / d) ** 2 + 0.3
    assert np.allclose(p["mean2d"][0], [64.0, 48.0], atol=1e-12)
    assert np.allclose(p["conic"][0], [1 / sig2, 0.0, 1 / sig2], rtol=1e-12)
    assert p["radius"][0] == math.ceil(3 * math.sqrt(sig2 + math.sqrt(0.1)))
    assert abs(p["depth"][0] - d) < 1e-12


def test_rotated_anisotropic_conic():
    """Scales (s1, s2, s3) turned by phi about the optical axis, at the centre:
    Sigma' = (f/d)^2 R(phi) diag(s1^2, s2^2) R(phi)^T + 0.3 I."""
    f, d, phi = 80.0, 5.0, 0.6
    s = np.array([0.12, 0.04, 0.3])
    cam = axis_camera(W=128, H=128, f=f, dist=d)
    q = [math.cos(phi / 2), 0, 0, math.sin(phi / 2)]
    g = one_gaussian([0, 0, 0], np.log(s), q, 0.0, [0.5] * 3)
    p = oracle.project(g, cam)
    R2 = np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])
    S = (f / d) ** 2 * R2 @ np.diag(s[:2] ** 2) @ R2.T + 0.3 * np.eye(2)
    K = np.linalg.inv(S)
    assert np.allclose(p["conic"][0], [K[0, 0], K[0, 1], K[1, 1]], rtol=1e-12)


def test_off_axis_isotropic_projection():
    """Isotropic Gaussian at camera-space (x, y, z): mean2d = f (x, y)/z + c and
    Sigma' = s^2 J J^T + 0.3 I with J the pinhole Jacobian."""
    f, s = 90.0, 0.07
    x, y, z = 0.6, -0.4, 3.0
    cam = axis_camera(W=160, H=120, f=f, dist=0.0)
    g = one_gaussian([x, y, z], [math.log(s)] * 3, [1, 0, 0, 0], 0.0, [0.5] * 3)
    p = oracle.project(g, cam)
    assert np.allclose(p["mean2d"][0], [f * x / z + 80, f * y / z + 60], rtol=1e-13)
    J = np.array([[f / z, 0, -f * x / z**2], [0, f / z, -f * y / z**2]])
    S = s * s * J @ J.T + 0.3 * np.eye(2)
    K = np.linalg.inv(S)
    assert np.allclose(p["conic"][0], [K[0, 0], K[0, 1], K[1, 1]], rtol=1e-12)


def test_frustum_guard_clamps_jacobian():
    """Beyond 1.3 tan(fov/2) the Jacobian uses the clamped ratio, the centre does not."""
    f, s, z = 64.0, 0.5, 2.0
    W = 64
    lim = 1.3 * W / (2 * f)
    x = 1.0 * z  # x/z = 1.0 > lim = 0.65
    cam = axis_camera(W=W, H=64, f=f, dist=0.0)
    g = one_gaussian([x, 0, z], [math.log(s)] * 3, [1, 0, 0, 0], 0.0, [0.5] * 3)
    p = oracle.project(g, cam)
    J = np.array([[f / z, 0, -f * lim / z], [0, f / z, 0]])
    S = s * s * J @ J.T + 0.3 * np.eye(2)
    K = np.linalg.inv(S)
    assert np.allclose(p["conic"][0], [K[0, 0], K[0, 1], K[1, 1]], rtol=1e-12)
    assert abs(p["mean2d"][0][0] - (f * x / z + 32)) < 1e-12


def test_near_plane_and_offscreen_cull():
    cam = axis_camera(dist=0.0)
    g = concat([
        one_gaussian([0, 0, 0.1], [-3] * 3, [1, 0, 0, 0], 0.0, [0.5] * 3),  # behind near
        one_gaussian([50, 0, 1.0], [-3] * 3, [1, 0, 0, 0], 0.0, [0.5] * 3),  # far off screen
        one_gaussian([0, 0, 1.0], [-3] * 3, [1, 0, 0, 0], 0.0, [0.5] * 3),  # visible
    ])
    p = oracle.project(g, cam)
    assert list(p["visible"]) == [0, 0, 1]


def test_tile_rect_definition():
    """The rectangle holds exactly the tiles whose span meets [m - r, m + r]."""
    rng = np.random.default_rng(0)
    W, H = 200, 120
    for _ in range(300):
        m = rng.uniform(-40, 240, 2)
        r = int(rng.integers(1, 40))
        ranges, lst = oracle.bin_sort(m[None], [r], [1.0], [1], W, H)
        TW, TH = (W + 15) // 16, (H + 15) // 16
        for ty in range(TH):
            for tx in range(TW):
                meets = (16 * tx <= m[0] + r and 16 * tx + 16 > m[0] - r and
                         16 * ty <= m[1] + r and 16 * ty + 16 > m[1] - r)
                t = ty * TW + tx
                assert (ranges[t, 1] - ranges[t, 0] == 1) == meets


# ---------------------------------------------------------------- blending
def test_centred_pixel_value_closed_form():
    """A single isotropic Gaussian over black: pixel value = c min(0.99, o exp(-rho^2 / (2 sigma^2)))
    (or 0 when that is below 1/255), T = 1 - alpha."""
    f, s, d = 64.0, 0.08, 4.0
    W = H = 64
    cam = axis_camera(W=W, H=H, f=f, dist=d)
    o = 0.8
    c = np.array([0.9, 0.4, 0.2])
    g = one_gaussian([0, 0, 0], [math.log(s)] * 3, [1, 0, 0, 0], logit(o), c)
    out = oracle.render(g, [cam])
    sig2 = (f * s / d) ** 2 + 0.3
    r = math.ceil(3 * math.sqrt(sig2 + math.sqrt(0.1)))
    for v in range(H):
        for u in range(W):
            rho2 = (u + 0.5 - 32) ** 2 + (v + 0.5 - 32) ** 2
            a = min(0.99, o * math.exp(-rho2 / (2 * sig2)))
            inside = abs(u + 0.5 - 32) <= r + 16 and abs(v + 0.5 - 32) <= r + 16
            tile_ok = (16 * (u // 16) <= 32 + r and 16 * (u // 16) + 16 > 32 - r and
                       16 * (v // 16) <= 32 + r and 16 * (v // 16) + 16 > 32 - r)
            if a < 1 / 255 or not tile_ok:
                a = 0.0
            assert inside or a == 0.0
            assert np.allclose(out["rgb"][0][:, v, u], c * a, atol=1e-14)
            assert abs(out["T"][0][v, u] - (1 - a)) < 1e-14


def test_telescoping_identity_and_importance_total():
    """With every colour 1 and a black background, C = sum_i a_i T_i, so
    C + T_final = 1 per pixel, and the importance weights sum to sum C."""
    g, cams = synthetic.plain_forward_scene()
    g = synthetic.widen(g)
    g["sh"] = np.full_like(g["sh"], (1.0 - 0.5) * 2 * math.sqrt(math.pi))
    out = oracle.render(g, cams)
    C, T = out["rgb"][0], out["T"][0]
    assert np.abs(C[0] + T - 1).max() < 1e-12
    assert abs(out["importance_w"].sum() - C[0].sum()) < 1e-9 * C[0].sum()
    assert (C[0] > 0.5).mean() > 0.05  # the scene is not empty


def test_alpha_threshold_straddle():
    """o G just above 1/255 blends, just below does not."""
    f, s, d = 64.0, 0.08, 4.0
    cam = axis_camera(W=32, H=32, f=f, dist=d)
    sig2 = (f * s / d) ** 2 + 0.3
    # pixel (16, 16) centre is at (16.5, 16.5); the Gaussian sits at (16, 16)
    rho2 = 0.5
    G = math.exp(-rho2 / (2 * sig2))
    for factor, blended in ((1.001, True), (0.999, False)):
        o = factor * (1 / 255) / G
        g = one_gaussian([0, 0, 0], [math.log(s)] * 3, [1, 0, 0, 0], logit(o), [1, 1, 1])
        out = oracle.render(g, [cam])
        val = out["rgb"][0][0, 16, 16]
        if blended:
            assert abs(val - o * G) < 1e-15 and out["n_contrib"][0][16, 16] == 1
        else:
            assert val == 0.0 and out["n_contrib"][0][16, 16] == 0


def test_alpha_clamp_at_099():
    cam = axis_camera(W=32, H=32, f=64.0, dist=4.0)
    # centre the Gaussian on the pixel centre (16.5, 16.5): world x = 0.5 * d / f
    x = 0.5 * 4.0 / 64.0
    g = one_gaussian([x, x, 0], [math.log(0.08)] * 3, [1, 0, 0, 0], logit(0.999), [1, 1, 1])
    out = oracle.render(g, [cam])
    assert abs(out["rgb"][0][0, 16, 16] - 0.99) < 1e-15
    assert abs(out["T"][0][16, 16] - 0.01) < 1e-15


def test_termination_stack():
    """Four identical Gaussians with alpha 0.95 at one pixel: T goes
    1 -> 0.05 -> 0.0025 -> 1.25e-4; the fourth would leave 6.25e-6 < 1e-4,
    so it is not blended and the pixel stops with three contributors."""
    cam = axis_camera(W=32, H=32, f=64.0, dist=4.0)
    cam["cx"] = cam["cy"] = 16.5  # the optical axis passes through pixel (16, 16)'s centre
    gs = [one_gaussian([0, 0, 0.01 * k], [math.log(0.08)] * 3, [1, 0, 0, 0], logit(0.95), [1, 1, 1]) for k in range(4)]
    out = oracle.render(concat(gs), [cam])
    assert out["n_contrib"][0][16, 16] == 3
    assert abs(out["T"][0][16, 16] - 0.05**3) < 1e-15
    assert abs(out["rgb"][0][0, 16, 16] - (1 - 0.05**3)) < 1e-14
    assert list(out["importance_cnt"]) == [int(c) for c in out["importance_cnt"]]


def test_depth_near_ties_flag_the_pixels_they_decide():
    """Two list entries closer in depth than a single-precision key resolves
    (relative 1e-8) are flagged at a pixel where both blend (their order
    changes the blend) or where one of them is the pixel's last blended entry
    (its position is n_contrib); 1e-3 apart they are not; a near tie of two
    entries too faint to blend, or of a blended entry that is not the last, moves
    no output and is not flagged."""
    cam = axis_camera(W=32, H=32, f=64.0, dist=4.0)
    cam["cx"] = cam["cy"] = 16.5

    def pair(dz, p_front, p_back):
        # centres a little off the pixel centre, so that no power sits at 0
        return concat([one_gaussian([0.02, 0, 0.0], [math.log(0.08)] * 3, [1, 0, 0, 0], logit(p_front), [1, 0, 0]),
                       one_gaussian([0.02, 0, dz], [math.log(0.08)] * 3, [1, 0, 0, 0], logit(p_back), [0, 1, 0])])

    assert oracle.render(pair(4e-8, 0.5, 0.5), [cam])["ambig"][0][16, 16]      # both blend
    assert oracle.render(pair(4e-8, 0.5, 0.001), [cam])["ambig"][0][16, 16]    # the last blended entry's position
    assert not oracle.render(pair(4e-3, 0.5, 0.5), [cam])["ambig"][0][16, 16]  # resolved in single precision
    assert not oracle.render(pair(4e-8, 0.001, 0.001), [cam])["ambig"][0][16, 16]  # neither blends
    # a blended entry tied with a faint one, then another blended entry: the
    # tie moves no output of the pixel (n_contrib is the later entry's)
    later = one_gaussian([0.02, 0, 0.1], [math.log(0.08)] * 3, [1, 0, 0, 0], logit(0.5), [0, 0, 1])
    g3 = concat([pair(4e-8, 0.5, 0.001), later])
    out = oracle.render(g3, [cam])
    assert out["n_contrib"][0][16, 16] == 3 and not out["ambig"][0][16, 16]


def test_permutation_invariance():
    g, cams = synthetic.plain_forward_scene()
    g = synthetic.widen(g)
    rng = np.random.default_rng(9)
    perm = rng.permutation(g["means"].shape[0])
    gp = dict(g)
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        gp[k] = g[k][perm]
    a = oracle.render(g, cams)
    b = oracle.render(gp, cams)
    # all depths distinct in this scene, so the per-tile orders agree
    assert len(np.unique(g["means"][:, 2])) == g["means"].shape[0]
    assert np.array_equal(a["rgb"][0], b["rgb"][0])
    assert np.array_equal(a["T"][0], b["T"][0])
    assert np.array_equal(a["n_contrib"][0], b["n_contrib"][0])
    assert np.allclose(a["importance_w"][perm], b["importance_w"], rtol=0, atol=1e-12)
    assert np.array_equal(a["importance_cnt"][perm], b["importance_cnt"])


def brute_force(g, cam, settings=oracle.DEFAULT_SETTINGS):
    """Per pixel: every Gaussian whose tile rectangle holds the pixel's tile,
    sorted by (depth, index), blended front to back -- no tile lists."""
    p = oracle.project(g, cam)
    W, H = cam["width"], cam["height"]
    N = len(p["depth"])
    img = np.zeros((3, H, W))
    Tm = np.ones((H, W))
    for v in range(H):
        for u in range(W):
            tx, ty = u // 16, v // 16
            cand = [i for i in range(N) if p["visible"][i] and p["rect"][i][0] <= tx < p["rect"][i][2]
                    and p["rect"][i][1] <= ty < p["rect"][i][3]]
            cand.sort(key=lambda i: (p["depth"][i], i))
            T = 1.0
            C = np.zeros(3)
            for i in cand:
                dx = p["mean2d"][i][0] - (u + 0.5)
                dy = p["mean2d"][i][1] - (v + 0.5)
                A, B, Cc = p["conic"][i]
                power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy
                if power > 0:
                    continue
                a = min(settings["alpha_max"], p["opacity"][i] * math.exp(power))
                if a < settings["alpha_min"]:
                    continue
                if T * (1 - a) < settings["T_min"]:
                    break
                C += p["rgb"][i] * a * T
                T *= 1 - a
            img[:, v, u] = C
            Tm[v, u] = T
    return img, Tm


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_brute_force_equals_tiled(seed):
    g = synthetic.widen(synthetic.gaussians(16, seed, mean_mode="uniform", mean_scale=(1, 1, 1),
                                            log_scale=(-2.3, 0.4), sh_degree=2, sh_std=0.3))
    cam = axis_camera(W=32, H=32, f=32.0, dist=3.0)
    out = oracle.render(g, [cam])
    img, T = brute_force(g, cam)
    assert np.abs(out["rgb"][0] - img).max() < 1e-13
    assert np.abs(out["T"][0] - T).max() < 1e-13


def test_background_adds_T_bg():
    g, cams = synthetic.plain_forward_scene()
    g = synthetic.widen(g)
    a = oracle.render(g, cams)
    b = oracle.render(g, cams, bg=(0.2, 0.5, 1.0))
    for ch, bgc in enumerate((0.2, 0.5, 1.0)):
        assert np.abs(b["rgb"][0][ch] - (a["rgb"][0][ch] + a["T"][0] * bgc)).max() < 1e-13


# ---------------------------------------------------------------- decode / apply
def quat_mat(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_decode_endpoints_exact():
    lo = np.array([-0.08, -0.08, -0.08, 0.99, -0.08, -0.08, -0.08])
    hi = np.array([0.08, 0.08, 0.08, 1.0, 0.08, 0.08, 0.08])
    m = np.zeros((7, 1, 2), np.uint16)
    m[:, 0, 1] = 65535
    base_m = np.zeros((2, 3))
    base_q = np.tile([1.0, 0, 0, 0], (2, 1))
    om, oq = oracle.decode_apply(m, lo, hi, base_m, base_q, quat_mode=oracle.QUAT_ADD)
    assert np.array_equal(om[0], lo[:3]) and np.array_equal(om[1], hi[:3])
    assert np.array_equal(oq[0], base_q[0] + lo[3:]) and np.array_equal(oq[1], base_q[1] + hi[3:])


def test_decode_identity_rotation_keeps_quat():
    rng = np.random.default_rng(1)
    N = 50
    lo = np.array([-0.08] * 3 + [0.0] + [-1.0] * 3)
    hi = np.array([0.08] * 3 + [1.0] + [1.0] * 3)
    m = np.zeros((7, 8, 8), np.uint16)
    m[3] = 65535  # w = 1
    m[4:7] = 32767  # x, y, z = -1 + 2 * 32767/65535 ~ -1.5e-5
    m[4:7] += 0  # keep
    base_q = rng.standard_normal((N, 4))
    base_q /= np.linalg.norm(base_q, axis=1, keepdims=True)
    _, oq = oracle.decode_apply(m, lo, hi, rng.standard_normal((N, 3)), base_q)
    # the decoded delta is within 2e-5 of identity
    assert np.abs(np.abs(np.sum(oq * base_q, axis=1)) - 1).max() < 1e-8


def test_decode_compose_two_frames_equals_product():
    """Frame updates applied in turn (d_t) equal the composed rotation applied
    to the anchor (D_t); as matrices R(dq2 (x) dq1 (x) q) = R(dq2) R(dq1) R(q)."""
    N = 64
    m1, lo, hi = synthetic.update_map(N, 1001, size=8)
    m2, _, _ = synthetic.update_map(N, 1002, size=8)
    rng = np.random.default_rng(2)
    base_m = rng.standard_normal((N, 3))
    base_q = rng.standard_normal((N, 4))
    mA, qA = oracle.decode_apply(m1, lo, hi, base_m, base_q)
    mB, qB = oracle.decode_apply(m2, lo, hi, mA, qA)
    z = np.zeros((N, 3))
    ident = np.tile([1.0, 0, 0, 0], (N, 1))
    _, d1 = oracle.decode_apply(m1, lo, hi, z, ident)
    d2m, d2 = oracle.decode_apply(m2, lo, hi, z, ident)
    d1m, _ = oracle.decode_apply(m1, lo, hi, z, ident)
    for i in range(N):
        assert np.allclose(quat_mat(qB[i]), quat_mat(d2[i]) @ quat_mat(d1[i]) @ quat_mat(base_q[i]), atol=1e-12)
    assert np.allclose(mB, base_m + d1m + d2m, atol=1e-15)


def test_decode_rejects_too_many_gaussians():
    with pytest.raises(ValueError):
        oracle.decode_apply(np.zeros((7, 2, 2), np.uint16), np.zeros(7), np.ones(7), np.zeros((5, 3)),
                            np.zeros((5, 4)))


# ---------------------------------------------------------------- adjoint vs central differences
def fd_scene(seed):
    """Few Gaussians, moderate opacity (no alpha clamp), SH degree 3, two views;
    one large Gaussian outside the frustum guard in the first view."""
    rng = np.random.default_rng(seed)
    g = synthetic.widen(synthetic.gaussians(7, seed, mean_mode="uniform", mean_scale=(0.8, 0.8, 0.8),
                                            log_scale=(-1.9, 0.3), sh_degree=3, sh_std=0.25, opacity_std=0.5))
    g["opacity_logit"] = np.clip(g["opacity_logit"], -1.5, 1.2)  # o <= 0.77
    extra = one_gaussian([2.6, 0.1, 0.5], [math.log(0.6), math.log(0.3), math.log(0.4)], [0.9, 0.2, -0.3, 0.1],
                         0.3, [0.5] * 3, sh_degree=3)
    extra["sh"][0, 1:] = rng.normal(0, 0.2, (15, 3))
    g = concat([g, extra])
    cams = [synthetic.camera((0.0, 0.0, -3.0), 40, 36, fov_x_deg=55.0),
            synthetic.camera((1.2, -0.6, -2.8), 36, 40, fov_x_deg=60.0)]
    return g, cams


def loss_and_weights(g, cams, wts):
    out = oracle.render(g, cams)
    return sum(float((w * r).sum()) for w, r in zip(wts, out["rgb"])), out


@pytest.mark.parametrize("seed", [11, 12])
def test_adjoint_matches_central_differences(seed):
    g, cams = fd_scene(seed)
    rng = np.random.default_rng(seed + 100)
    wts = [rng.standard_normal((3, c["height"], c["width"])) for c in cams]
    L0, out = loss_and_weights(g, cams, wts)
    assert not any(a.any() for a in out["ambig"])
    # the guard case is exercised: the extra Gaussian is outside 1.3 tan(fov/2) in view 0
    lim = 1.3 * cams[0]["width"] / (2 * cams[0]["fx"])
    assert 2.6 / 3.5 > lim
    grads = oracle.render_backward(g, cams, wts)
    assert np.abs(grads["means"][-1]).max() > 1e-3  # the guarded Gaussian is blended
    h = 1e-6
    checked = 0
    for key in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        arr = g[key]
        flat = arr.reshape(-1)
        gflat = grads[key].reshape(-1)
        idx = range(flat.size) if key != "sh" else rng.choice(flat.size, 60, replace=False)
        for j in idx:
            orig = flat[j]
            flat[j] = orig + h
            Lp, _ = loss_and_weights(g, cams, wts)
            flat[j] = orig - h
            Lm, _ = loss_and_weights(g, cams, wts)
            flat[j] = orig
            fd = (Lp - Lm) / (2 * h)
            scale = max(1.0, abs(fd))
            assert abs(fd - gflat[j]) < 2e-6 * scale, (key, j, fd, gflat[j])
            checked += 1
    assert checked > 100


def test_adjoint_zero_where_alpha_clamped():
    """Where o G > 0.99 alpha is the constant 0.99, so a loss on that pixel
    alone passes no gradient to the opacity or the position."""
    cam = axis_camera(W=16, H=16, f=16.0, dist=4.0)
    x = 0.5 * 4.0 / 16.0
    g = one_gaussian([x, x, 0], [math.log(0.02)] * 3, [1, 0, 0, 0], logit(0.9999), [1, 1, 1])
    out = oracle.render(g, [cam])
    assert out["importance_cnt"][0] >= 1
    # the loss reads only the pixel under the centre, where o G = 0.9999
    w = np.zeros((3, 16, 16))
    w[:, 8, 8] = 1.0
    grads = oracle.render_backward(g, [cam], [w])
    assert grads["opacity_logit"][0] == 0.0
    assert np.all(grads["means"] == 0.0)
    # elsewhere alpha is not clamped and the gradient is not zero
    w2 = np.zeros((3, 16, 16))
    w2[:, 8, 9] = 1.0
    assert oracle.render_backward(g, [cam], [w2])["opacity_logit"][0] != 0.0


def test_l1_gradient_sign_and_scale():
    r = [np.array([[[0.5, 0.2]], [[0.1, 0.1]], [[0.0, 1.0]]])]
    t = [np.array([[[0.4, 0.2]], [[0.3, 0.1]], [[0.0, 0.5]]])]
    loss, gr = oracle.l1_loss_grad(r, t)
    assert abs(loss - (0.1 + 0.2 + 0.5) / 6) < 1e-15
    assert np.array_equal(np.sign(gr[0]), [[[1, 0]], [[-1, 0]], [[0, 1]]])
    assert np.allclose(np.abs(gr[0])[gr[0] != 0], 1 / 6)


# ---------------------------------------------------------------- densification statistic
def test_densification_statistic_per_view_norms_and_binned_views():
    """Sec. III-B densifies where the view-space positional gradient is large;
    the statistic is the sum over views of |dL/d mean2d| with the count of views
    in which the Gaussian is binned.  One Gaussian, five cameras:
      A, B  see it from different directions (random linear loss on both),
      C     has it behind the camera (culled),
      D     has it in front but off the image (no tile: not binned),
      E     bins it, but the loss has no weight there (zero gradient, still a view).
    dL/d mean2d of a view is pinned without the adjoint: shifting that camera's
    principal point by h moves only that view's projected centre by h (mean2d =
    f t/z + c), so a central difference of the forward loss in cx / cy gives it.
    The statistic must be |v_A| + |v_B| (not |v_A + v_B|), the count 3 (A, B, E)."""
    g = one_gaussian([0.1, -0.05, 0.2], [math.log(0.12), math.log(0.08), math.log(0.1)],
                     [0.9, 0.3, -0.2, 0.25], logit(0.6), [0.8, 0.3, 0.5])
    cams = [synthetic.camera((0.0, 0.0, -3.0), 40, 36, fov_x_deg=50.0),           # A
            synthetic.camera((2.2, -1.0, -1.6), 36, 40, fov_x_deg=55.0),          # B
            synthetic.camera((0.0, 0.0, 3.0), 32, 32, fov_x_deg=50.0, target=(0.0, 0.0, 6.0)),   # C
            synthetic.camera((0.0, 0.0, -3.0), 32, 32, fov_x_deg=30.0, target=(4.0, 0.0, 0.0)),  # D
            synthetic.camera((-1.5, 0.5, -2.5), 30, 30, fov_x_deg=50.0)]          # E
    vis = [oracle.project(g, c) for c in cams]
    assert [bool(p["visible"][0]) for p in vis] == [True, True, False, False, True]
    assert vis[3]["depth"][0] > cams[3]["near"]  # D: in front of the camera, yet not binned
    rng = np.random.default_rng(5)
    wts = [rng.standard_normal((3, c["height"], c["width"])) for c in cams]
    wts[4][:] = 0.0
    L0, out = loss_and_weights(g, cams, wts)
    assert not any(a.any() for a in out["ambig"])
    h = 1e-6
    v = []
    for k, c in enumerate(cams):
        comp = []
        for key in ("cx", "cy"):
            cp = [dict(x) for x in cams]
            cp[k][key] = c[key] + h
            Lp, _ = loss_and_weights(g, cp, wts)
            cp[k][key] = c[key] - h
            Lm, _ = loss_and_weights(g, cp, wts)
            comp.append((Lp - Lm) / (2 * h))
        v.append(np.array(comp))
    assert np.linalg.norm(v[0]) > 1e-2 and np.linalg.norm(v[1]) > 1e-2
    assert all(np.abs(v[k]).max() == 0.0 for k in (2, 3, 4))
    want = np.linalg.norm(v[0]) + np.linalg.norm(v[1])
    # the two readings differ clearly on this scene
    assert abs(want - np.linalg.norm(v[0] + v[1])) > 0.05 * want
    got = oracle.render_backward(g, cams, wts, densify=True)
    assert abs(got["densify_grad"][0] - want) < 1e-6 * max(1.0, want), (got["densify_grad"][0], want)
    assert int(got["densify_views"][0]) == 3


# ---------------------------------------------------------------- the OpenMP timing build of the oracle
def test_openmp_timing_build_computes_the_oracle():
    """The benchmark times the oracle on all host cores through a separate
    OpenMP build of the same source: its forward must equal the oracle's bit
    for bit and its adjoint up to the order of additions."""
    from oracle import timing
    g, cams = fd_scene(21)
    cams = cams + [synthetic.camera((0.4, 0.3, -3.2), 53, 37, fov_x_deg=50.0)]
    ref = oracle.render(g, cams)
    got = timing.render(g, cams)
    for v in range(len(cams)):
        assert np.array_equal(got["rgb"][v], ref["rgb"][v])
        assert np.array_equal(got["T"][v], ref["T"][v])
        assert np.array_equal(got["n_contrib"][v], ref["n_contrib"][v])
    assert got["pairs"] == ref["pairs"]
    assert np.array_equal(got["importance_cnt"], ref["importance_cnt"])
    assert np.allclose(got["importance_w"], ref["importance_w"], rtol=1e-12, atol=1e-15)
    rng = np.random.default_rng(4)
    dL = [rng.standard_normal((3, c["height"], c["width"])) for c in cams]
    gr, gw = oracle.render_backward(g, cams, dL), timing.render_backward(g, cams, dL)
    for k in gr:
        assert np.allclose(gw[k], gr[k], rtol=1e-10, atol=1e-12 * np.abs(gr[k]).max()), k
    assert timing.threads() >= 1
