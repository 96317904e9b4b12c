"""Adaptive pruning of streamed deltas (Sec. III-C, Algorithm 1).

The dense pruning-level space S_t^d lists, for pruning levels 0 %, 10 %, ...,
100 % of the Gaussians (lowest usage frequency first), the reconstruction
quality and the transmitted size of the pruned delta d'_t = p(D_t - D'_{t-1}).
Algorithm 1 keeps the levels before the first quality "cliff" (a drop more
than beta times the previous drop) and binary-searches that candidate list,
whose sizes decrease with the level, for the lowest level whose size fits the
per-frame budget B / R.

Quality is the PSNR of the pruned frame against the unpruned one, rendered by
the library for a set of views; every rendering, pruning, delta and error step
runs in libairgs kernels.  Only the level loop and Algorithm 1 (a few
comparisons) run on the host.

Readings where the listing is silent: a previous drop of exactly 0 makes any
later quality loss a cliff; when no candidate level fits the budget the result
is the cliff level if a cliff was found, else the last candidate (the most
pruning the candidates allow).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from ._abi import AIRGS_DELTA_ANCHOR

UPDATE_CHANNELS = 7  # position offset (3) + rotation delta (4) per Gaussian (Sec. III-B, Eq. 3)
BYTES_PER_GAUSSIAN = UPDATE_CHANNELS * 2  # seven 16-bit channels per Gaussian in the update maps
BETA = 2.0  # the cliff multiplier beta of Algorithm 1 as the experiments set it (Sec. V)


@dataclass
class Level:
    fraction: float   # fraction of Gaussians pruned
    quality: float    # PSNR (dB) against the unpruned frame
    size: int         # bytes of the transmitted delta


def _is_cliff(drop: float, previous: float, beta: float) -> bool:
    if previous == 0.0:
        return drop < 0.0
    return drop / previous > beta


def select_pruning_level(space, beta: float, bandwidth: float, frame_rate: float) -> int:
    """Algorithm 1: the pruning level (index into `space`, a list of
    (quality, size) pairs ordered by increasing pruning) for bandwidth B and
    target frame rate R."""
    q = [float(s[0]) for s in space]
    size = [float(s[1]) for s in space]
    if not q:
        raise ValueError("empty pruning-level space")
    candidates = [0]
    cliff = None
    if len(q) > 1:
        previous = q[1] - q[0]
        for i in range(1, len(q)):
            drop = q[i] - q[i - 1]
            if _is_cliff(drop, previous, beta):
                cliff = i
                break
            candidates.append(i)
            previous = drop
    budget = bandwidth / frame_rate
    chosen = cliff if cliff is not None else candidates[-1]
    lo, hi = 0, len(candidates) - 1
    while lo <= hi:
        mid = (lo + hi) // 2
        level = candidates[mid]
        if size[level] <= budget:
            chosen = level
            hi = mid - 1
        else:
            lo = mid + 1
    return chosen


def psnr(sse: float, n_values: int) -> float:
    """PSNR of images in [0, 1] from their sum of squared differences."""
    if sse <= 0.0:
        return float("inf")
    return 10.0 * math.log10(n_values / sse)


def pruning_level_space(rast, D_t: torch.Tensor, D_sent: torch.Tensor, importance: torch.Tensor, cams,
                        fractions=tuple(i / 10 for i in range(11)), quat_add: bool = True):
    """Build S_t^d on the device.  D_t, D_sent: channel-major [7, n] cumulative
    delta and the record of what was transmitted; importance: [n] usage
    frequency.  The context `rast` holds the anchor GC_k; frames are
    reconstructed as GC_k + D'_t.  Returns [Level], the unpruned image first
    rendered as reference.  D_sent is not modified."""
    n = D_t.shape[1]
    rast.apply_frame_delta(D_t, mode=AIRGS_DELTA_ANCHOR, quat_add=quat_add)
    ref = rast.render(cams).rgb
    total_px = sum(3 * int(c["width"]) * int(c["height"]) for c in cams)
    out = []
    for f in fractions:
        n_prune = int(round(f * n))
        keep = rast.prune_mask(importance, n_prune)
        record = D_sent.clone()
        _, nonzero = rast.prune_delta(D_t, record, keep)
        rast.apply_frame_delta(record, mode=AIRGS_DELTA_ANCHOR, quat_add=quat_add)
        img = rast.render(cams).rgb
        sse = float(np.sum(rast.image_sse(cams, img, ref).cpu().numpy()))
        sent = int(nonzero.cpu()[0])  # Gaussians with a non-zero transmitted delta
        out.append(Level(fraction=f, quality=psnr(sse, total_px), size=sent * BYTES_PER_GAUSSIAN))
    return out
