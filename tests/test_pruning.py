"""Usage-frequency pruning p(.) and pruning-level selection (Sec. III-C,
Algorithm 1): Algorithm 1 against a linear-scan restatement (its hand-worked
cases are fixtures under tests/golden/, checked by test_golden.py), the
oracle's p(.) / record update against their definitions, and the CUDA kernels
against the oracle."""
import math

import numpy as np
import pytest

import oracle
import synthetic
from paper_2512_20943_b300.pruning import psnr, select_pruning_level


# ---------------------------------------------------------------- Algorithm 1 (host)
def _linear_reference(space, beta, B, R):
    """The same selection by a linear scan of the candidates."""
    q = [a for a, _ in space]
    cand, cliff, prev = [0], None, (q[1] - q[0] if len(q) > 1 else 0.0)
    for i in range(1, len(q)):
        drop = q[i] - q[i - 1]
        is_cliff = (drop < 0) if prev == 0 else (drop / prev > beta)
        if is_cliff:
            cliff = i
            break
        cand.append(i)
        prev = drop
    fits = [c for c in cand if space[c][1] <= B / R]
    if fits:
        return min(fits)
    return cliff if cliff is not None else cand[-1]


def test_algorithm1_binary_search_equals_linear_scan():
    rng = np.random.default_rng(0)
    for _ in range(2000):
        n = int(rng.integers(1, 12))
        drops = -np.abs(rng.normal(0.3, 0.3, n))
        drops[rng.random(n) < 0.15] *= 10  # occasional cliffs
        q = 35 + np.concatenate([[0.0], np.cumsum(drops[1:])])
        sizes = np.sort(rng.integers(1, 100, n))[::-1]  # size falls with pruning
        space = list(zip(q.tolist(), sizes.tolist()))
        B = float(rng.integers(1, 120))
        assert select_pruning_level(space, 2.0, B, 1.0) == _linear_reference(space, 2.0, B, 1.0)


def test_psnr():
    assert psnr(0.0, 10) == math.inf
    assert abs(psnr(3 * 100 * 1e-4, 3 * 100) - 40.0) < 1e-12


# ---------------------------------------------------------------- oracle p(.) pins
def test_oracle_prune_mask_order_and_ties():
    w = np.array([0.5, 0.1, 0.1, 0.0, 2.0, -1.0, np.nan, 0.1])
    # ascending, equal weights by index: -1 and NaN count as 0 -> order 3, 5, 6, 1, 2, 7, 0, 4
    keep = oracle.prune_mask(w, 4)
    assert list(np.nonzero(keep == 0)[0]) == [1, 3, 5, 6]
    assert oracle.prune_mask(w, 0).all() and not oracle.prune_mask(w, len(w)).any()


def test_oracle_record_tracks_transmitted_delta():
    """D'_t accumulates exactly what was sent, so a later unpruned frame sends
    the whole remaining difference (no cumulative pruning drift)."""
    rng = np.random.default_rng(1)
    n = 50
    D1 = rng.normal(size=(7, n))
    keep = oracle.prune_mask(rng.random(n), 20)
    d1, rec1 = oracle.prune_delta(D1, np.zeros((7, n)), keep)
    assert np.all(d1[:, keep == 0] == 0) and np.allclose(d1[:, keep == 1], D1[:, keep == 1])
    D2 = D1 + rng.normal(size=(7, n))
    d2, rec2 = oracle.prune_delta(D2, rec1, np.ones(n, np.uint8))
    assert np.allclose(rec2, D2) and np.allclose(d1 + d2, D2)


def test_oracle_apply_delta_matches_decode():
    n = 40
    m, lo, hi = synthetic.update_map(n, 1003, size=8)
    lo64, hi64 = lo.astype(np.float64), hi.astype(np.float64)
    u = m.reshape(7, -1)[:, :n].astype(np.float64)
    delta = lo64[:, None] + u * ((hi64 - lo64) / 65535.0)[:, None]
    rng = np.random.default_rng(2)
    bm, bq = rng.normal(size=(n, 3)), rng.normal(size=(n, 4))
    for qa in (False, True):
        a = oracle.apply_delta(bm, bq, delta, quat_add=qa)
        b = oracle.decode_apply(m, lo64, hi64, bm, bq, oracle.QUAT_ADD if qa else oracle.QUAT_COMPOSE)
        assert np.allclose(a[0], b[0], atol=1e-15) and np.allclose(a[1], b[1], atol=1e-15)


# ---------------------------------------------------------------- CUDA kernels vs oracle
@pytest.mark.gpu
def test_prune_mask_and_delta_match_oracle():
    import torch
    from paper_2512_20943_b300 import Rasterizer
    rast = Rasterizer()
    rng = np.random.default_rng(3)
    n = 100_003
    w = rng.gamma(0.5, 1.0, n).astype(np.float32)
    w[rng.random(n) < 0.2] = 0.0           # many equal (zero) weights
    w[rng.random(n) < 0.05] = w[0]          # and ties at a positive value
    wt = torch.from_numpy(w).cuda()
    for n_prune in (0, 1, 12345, n // 2, n):
        keep = rast.prune_mask(wt, n_prune).cpu().numpy()
        assert np.array_equal(keep, oracle.prune_mask(w, n_prune)), n_prune
    D = rng.normal(size=(7, n)).astype(np.float32)
    rec = rng.normal(size=(7, n)).astype(np.float32)
    keep = oracle.prune_mask(w, n // 3)
    Dt, rect = torch.from_numpy(D).cuda(), torch.from_numpy(rec.copy()).cuda()
    d, nz = rast.prune_delta(Dt, rect, torch.from_numpy(keep).cuda())
    torch.cuda.synchronize()
    d_ref, rec_ref = oracle.prune_delta(D, rec, keep)
    assert np.abs(d.cpu().numpy() - d_ref).max() < 1e-6 and np.abs(rect.cpu().numpy() - rec_ref).max() < 1e-6
    assert int(nz.cpu()[0]) == int(((d_ref != 0).any(axis=0)).sum())


@pytest.mark.gpu
def test_apply_frame_delta_and_sse_match_oracle():
    import torch
    from paper_2512_20943_b300 import AIRGS_DELTA_ANCHOR, Rasterizer
    from tests._helpers import params, to_cuda
    g, cams = synthetic.plain_forward_scene()
    n = g["means"].shape[0]
    rast = Rasterizer()
    rast.set_anchor(*params(to_cuda(g)))
    delta = np.random.default_rng(4).normal(0, 0.01, (7, n)).astype(np.float32)
    delta[3] += 1.0
    for qa in (False, True):
        rast.apply_frame_delta(torch.from_numpy(delta).cuda(), mode=AIRGS_DELTA_ANCHOR, quat_add=qa)
        means, quats = (x.cpu().numpy() for x in rast.frame_state())
        rm, rq = oracle.apply_delta(g["means"], g["quats"], delta, quat_add=qa)
        assert np.abs(means - rm).max() < 1e-6 and np.abs(quats - rq).max() < 2e-6
    a = rast.render(cams).rgb
    b = torch.rand_like(a)
    sse = rast.image_sse(cams, a, b).cpu().numpy()
    assert abs(sse[0] - float(((a.double() - b.double()) ** 2).sum())) < 1e-9 * sse[0]


@pytest.mark.gpu
def test_pruning_level_space_and_selection():
    import torch
    from paper_2512_20943_b300 import Rasterizer
    from paper_2512_20943_b300.pruning import BYTES_PER_GAUSSIAN, pruning_level_space
    from tests._helpers import params, to_cuda
    g, cams = synthetic.per_frame_training_scene(n=20000, n_views=3, width=320, height=240)
    n = g["means"].shape[0]
    rast = Rasterizer()
    rast.set_anchor(*params(to_cuda(g)))
    w, _ = rast.gaussian_importance(cams)
    D = np.random.default_rng(5).normal(0, 0.01, (7, n)).astype(np.float32)
    space = pruning_level_space(rast, torch.from_numpy(D).cuda(), torch.zeros(7, n, device="cuda"), w, cams)
    assert len(space) == 11
    assert space[0].quality == math.inf and space[0].size == n * BYTES_PER_GAUSSIAN
    assert space[-1].size == 0
    sizes = [lv.size for lv in space]
    assert sizes == sorted(sizes, reverse=True)
    q = [min(lv.quality, 200.0) for lv in space]
    assert q[-1] < q[1]  # pruning everything costs quality
    lvl = select_pruning_level([(min(lv.quality, 200.0), lv.size) for lv in space], 2.0, 0.5 * space[0].size, 1.0)
    assert space[lvl].size <= 0.5 * space[0].size or lvl == len(space) - 1
