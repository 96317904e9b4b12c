"""Pins of the oracle's densification step (clone / split / discard, Sec. III-B;
the clone and split rules of 3D Gaussian Splatting's adaptive density control).

Each test fixes the result from something other than the oracle's own code:
hand-worked decisions at both thresholds, closed forms of the children's means
for an identity and a 90-degree rotation, the sample covariance of many
children against the Gaussian's covariance R S^2 R^T, and the scale division.
"""
import numpy as np
import pytest

import oracle


def _gaussians(log_scales, logits, quats=None, means=None, k=16):
    n = len(logits)
    rng = np.random.default_rng(11)
    return dict(means=np.zeros((n, 3)) if means is None else np.asarray(means, np.float64),
                log_scales=np.asarray(log_scales, np.float32).reshape(n, 3),
                quats=np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)) if quats is None else np.asarray(quats, np.float64),
                opacity_logit=np.asarray(logits, np.float32),
                sh=rng.normal(size=(n, k, 3)))


def test_decisions_at_both_thresholds():
    # size threshold 0.25: a largest log scale equal to float32(log 0.25) is not
    # large (clone); one float32 ulp above it is large (split).  Opacity 0.5:
    # logit 0 is alive, the next float32 below 0 is discarded.
    t = np.float32(np.log(0.25))
    up = np.nextafter(t, np.float32(1))
    small, large = [-3.0, -3.0, -3.0], [-3.0, float(up), -3.0]
    at = [float(t), -5.0, -4.0]
    neg0 = float(np.nextafter(np.float32(0), np.float32(-1)))
    cases = [  # (log_scales, logit, selected) -> (keep, clone, split)
        (small, 1.0, 0, (1, 0, 0)),
        (large, 1.0, 0, (1, 0, 0)),
        (small, 1.0, 1, (1, 1, 0)),
        (large, 1.0, 1, (0, 0, 1)),
        (at, 1.0, 1, (1, 1, 0)),
        (large, 0.0, 1, (0, 0, 1)),
        (large, neg0, 1, (0, 0, 0)),
        (small, neg0, 0, (0, 0, 0)),
        (small, -3.0, 1, (0, 0, 0)),
    ]
    g = _gaussians([c[0] for c in cases], [c[1] for c in cases])
    keep, clone, split = oracle.densify_classes(g["log_scales"], g["opacity_logit"], [c[2] for c in cases], 0.25, 0.5)
    got = np.stack([keep, clone, split], axis=1).astype(int)
    assert got.tolist() == [list(c[3]) for c in cases]
    # min_opacity 0 discards nothing, whatever the logit
    keep0, _, _ = oracle.densify_classes(g["log_scales"], np.full(len(cases), -80.0, np.float32), np.zeros(len(cases)),
                                         0.25, 0.0)
    assert keep0.all()


def test_output_layout_copies_and_parents():
    # Gaussians 0..5: keep, clone, split, discard, clone, split (in that order of roles)
    t = 0.25
    small, large = [-3.0, -3.0, -3.0], [-1.0, -3.0, -3.0]
    g = _gaussians([small, small, large, large, small, large], [2.0, 2.0, 2.0, -9.0, 2.0, 2.0],
                   means=np.arange(18, dtype=np.float64).reshape(6, 3))
    sel = [0, 1, 1, 1, 1, 1]
    z = np.random.default_rng(3).normal(size=(6, 2, 3))
    out = oracle.densify_apply(g, sel, z, t, 1.6, 0.01)
    # originals (unselected 0, cloned 1 and 4), copies (1, 4), children (2, 2, 5, 5)
    assert out["parent"].tolist() == [0, 1, 4, 1, 4, 2, 2, 5, 5]
    assert out["means"].shape == (9, 3) and out["sh"].shape == (9, 48)
    for j in range(5):  # originals and copies are the input rows unchanged
        p = out["parent"][j]
        assert np.array_equal(out["means"][j], g["means"][p])
        assert np.array_equal(out["log_scales"][j], g["log_scales"][p].astype(np.float64))
        assert np.array_equal(out["quats"][j], g["quats"][p])
        assert np.array_equal(out["sh"][j], g["sh"][p].reshape(-1))
    for j in range(5, 9):  # children keep rotation, opacity and SH
        p = out["parent"][j]
        assert np.array_equal(out["quats"][j], g["quats"][p])
        assert out["opacity_logit"][j] == np.float64(g["opacity_logit"][p])
        assert np.array_equal(out["sh"][j], g["sh"][p].reshape(-1))


def test_children_means_identity_rotation_closed_form():
    s = np.array([0.1, 0.2, 0.3])
    z = np.array([[[1.0, -2.0, 0.5], [0.0, 3.0, -1.0]]])
    for q in ([1.0, 0.0, 0.0, 0.0], [2.5, 0.0, 0.0, 0.0]):  # unnormalised quaternions are normalised first
        g = _gaussians([np.log(s)], [3.0], quats=[q], means=[[1.0, 2.0, 3.0]])
        out = oracle.densify_apply(g, [1], z, 0.01, 1.6)
        s32 = np.exp(np.float32(np.log(s)).astype(np.float64))
        want = np.array([1.0, 2.0, 3.0]) + s32 * z[0]
        np.testing.assert_allclose(out["means"], want, rtol=0, atol=1e-15)


def test_children_means_quarter_turn_closed_form():
    # q = (cos 45deg, 0, 0, sin 45deg): a quarter turn about z, R e_x = e_y and
    # R e_y = -e_x, so R (s * z) = (-s_y z_y, s_x z_x, s_z z_z)
    s = np.exp(np.float32(np.log([0.1, 0.2, 0.3])).astype(np.float64))
    c = np.sqrt(0.5)
    z = np.array([[[1.0, -2.0, 0.5], [0.25, 3.0, -1.0]]])
    g = _gaussians([np.log(s)], [3.0], quats=[[c, 0.0, 0.0, c]], means=[[0.0, 0.0, 0.0]])
    out = oracle.densify_apply(g, [1], z, 0.01, 1.6)
    for j in range(2):
        zx, zy, zz = z[0, j]
        np.testing.assert_allclose(out["means"][j], [-s[1] * zy, s[0] * zx, s[2] * zz], rtol=0, atol=1e-15)


def test_children_sample_the_gaussian_covariance():
    # the children of one Gaussian, split many times, scatter with covariance
    # Sigma = R S^2 R^T (the 3D Gaussian's covariance): sample estimate within 3 %
    m = 20000
    q = np.array([0.8, 0.3, -0.4, 0.2])
    log_s = np.log([0.05, 0.2, 0.6])
    g = _gaussians(np.tile(log_s, (m, 1)), np.full(m, 2.0), quats=np.tile(q, (m, 1)), k=1)
    z = np.random.default_rng(7).normal(size=(m, 2, 3))
    out = oracle.densify_apply(g, np.ones(m), z, 0.1, 1.6)
    assert out["means"].shape == (2 * m, 3)
    cov = np.cov(out["means"].T)
    qn = q / np.linalg.norm(q)
    w, x, y, zq = qn
    R = np.array([[1 - 2 * (y * y + zq * zq), 2 * (x * y - w * zq), 2 * (x * zq + w * y)],
                  [2 * (x * y + w * zq), 1 - 2 * (x * x + zq * zq), 2 * (y * zq - w * x)],
                  [2 * (x * zq - w * y), 2 * (y * zq + w * x), 1 - 2 * (x * x + y * y)]])
    S = np.diag(np.exp(np.float32(log_s).astype(np.float64)))
    sigma = R @ S @ S @ R.T
    assert np.linalg.norm(cov - sigma) < 0.03 * np.linalg.norm(sigma)
    # the transposed rotation scatters differently (the test can tell them apart)
    sigma_t = R.T @ S @ S @ R
    assert np.linalg.norm(cov - sigma_t) > 0.2 * np.linalg.norm(sigma)


@pytest.mark.parametrize("factor", [1.6, 2.0])
def test_children_scales_are_divided_by_the_split_factor(factor):
    log_s = np.float32(np.log([0.4, 0.5, 0.6]))
    g = _gaussians([log_s], [3.0])
    out = oracle.densify_apply(g, [1], np.zeros((1, 2, 3)), 0.1, factor)
    np.testing.assert_allclose(np.exp(out["log_scales"]), np.tile(np.exp(log_s.astype(np.float64)) / factor, (2, 1)),
                               rtol=1e-13)
    np.testing.assert_array_equal(out["means"], np.zeros((2, 3)))  # z = 0: children at the mean


def test_nothing_selected_or_all_discarded():
    g = _gaussians([[-3.0] * 3] * 4, [1.0, 1.0, 1.0, 1.0])
    out = oracle.densify_apply(g, np.zeros(4), np.zeros((4, 2, 3)), 0.25)
    assert out["parent"].tolist() == [0, 1, 2, 3]
    out = oracle.densify_apply(g, np.ones(4), np.zeros((4, 2, 3)), 0.25, 1.6, 0.9)
    assert out["parent"].tolist() == [] and out["means"].shape == (0, 3)
