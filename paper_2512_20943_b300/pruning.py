"""Adaptive pruning of streamed deltas (Sec. III-C, Algorithm 1).

The dense pruning-level space S_t^d lists, for pruning levels 0 %, 10 %, ...,
100 % of the Gaussians (lowest usage frequency first), the reconstruction
quality and the transmitted size of the pruned delta d'_t = p(D_t - D'_{t-1}).
The selection of Algorithm 1 admits the levels before the first quality
"cliff" (a drop more than beta times the drop before it) and returns the
least pruned admissible level whose size fits the per-frame budget B / R;
sizes do not increase with the level, so that level is found by bisection.

Quality is the PSNR of the pruned frame against the unpruned one, rendered by
the library for a set of views; every rendering, pruning, delta and error step
runs in libairgs kernels.  Only the level loop and Algorithm 1 (a few
comparisons) run on the host.

Readings where the section is silent: a previous drop of exactly 0 makes any
later quality loss a cliff; when no candidate level fits the budget the result
is the cliff level if a cliff was found, else the last candidate (the most
pruning the candidates allow).
"""
from __future__ import annotations

import bisect
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
    """A quality change is a cliff when it is more than beta times the drop
    before it (both changes are non-positive); after a flat step any loss is."""
    if previous == 0.0:
        return drop < 0.0
    return drop / previous > beta


def first_cliff(quality, beta: float):
    """Index of the first level whose quality change is a cliff relative to the
    change before it (the first change stands in for its own predecessor), or
    None when the space has no cliff."""
    changes = [b - a for a, b in zip(quality, quality[1:])]  # changes[k]: level k -> k + 1
    for k, change in enumerate(changes):
        if _is_cliff(change, changes[max(k - 1, 0)], beta):
            return k + 1
    return None


def select_pruning_level(space, beta: float, bandwidth: float, frame_rate: float) -> int:
    """Pruning level of Sec. III-C (Algorithm 1): `space` lists (quality, size)
    per level, ordered by increasing pruning, so sizes do not increase.  The
    admissible levels are those before the first quality cliff; of those, the
    result is the least pruned one whose transmitted size fits the per-frame
    budget B / R, located by bisection over the admissible sizes (a
    non-increasing sequence).  If no admissible level fits, the result is the
    cliff level when there is one, else the most pruned admissible level."""
    quality = [float(s[0]) for s in space]
    size = [float(s[1]) for s in space]
    if not quality:
        raise ValueError("empty pruning-level space")
    cliff = first_cliff(quality, beta)
    admissible = cliff if cliff is not None else len(quality)  # levels [0, admissible)
    budget = bandwidth / frame_rate
    # "fits the budget" goes from False to True along non-increasing sizes
    first_fit = bisect.bisect_left(range(admissible), True, key=lambda level: size[level] <= budget)
    if first_fit < admissible:
        return first_fit
    return cliff if cliff is not None else admissible - 1


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
    # every level is queued before any result is read back: one host wait for the space
    pending = []
    for f in fractions:
        n_prune = int(round(f * n))
        keep = rast.prune_mask(importance, n_prune)
        with torch.cuda.stream(rast.stream):  # freed in the library's stream order, read back or not
            record = D_sent.clone()
        _, nonzero = rast.prune_delta(D_t, record, keep)
        rast.apply_frame_delta(record, mode=AIRGS_DELTA_ANCHOR, quat_add=quat_add)
        img = rast.render(cams).rgb
        pending.append((f, rast.image_sse(cams, img, ref), nonzero))
    out = []
    for f, sse_v, nonzero in pending:
        sse = float(np.sum(sse_v.cpu().numpy()))
        sent = int(nonzero.cpu()[0])  # Gaussians with a non-zero transmitted delta
        out.append(Level(fraction=f, quality=psnr(sse, total_px), size=sent * BYTES_PER_GAUSSIAN))
    return out
