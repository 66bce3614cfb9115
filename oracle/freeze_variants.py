"""Freeze strategies of the ablation study (Sec. 5, "Freezing strategies"
and "Gradient information"; Table 3), written out plainly (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): imported by tests and
the benchmark's reference arm, never by the product path.

The paper compares its freeze rule (Eq. 4) with three variants:

* *random*: freeze 25% of the Gaussians at random;
* *mingrad*: freeze the 25% with the lowest gradients;
* *GSta-rgb*: the rule with the positional criterion only.

Readings (the paper gives no more detail):

* a Gaussian is eligible at an update when it is not frozen and was seen in
  the window (cnt > 0) -- the set the rule itself decides on;
* random: each eligible Gaussian is frozen independently with probability
  `fraction`, from a uniform draw u[i] in [0, 1) per Gaussian that the
  caller supplies (frozen when u[i] < fraction);
* mingrad: "gradient" is the rule's own measure, the larger of the two
  window averages in units of their thresholds,
  score = max(avg_xyz / eps_xyz, avg_rgb / eps_rgb); the
  k = floor(fraction * m) eligible Gaussians with the smallest
  (score, index) are frozen, m the eligible count (so only the rank cut
  differs from the rule, which freezes exactly where score < 1);
* every strategy then does what an Eq. 4 update does: the map only grows
  and the window statistics restart.

Averages, scores and comparisons are float32 operations (each one rounded),
the same numbers the rule compares; k is floor of the double product.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import planted

RULE, XYZ, RANDOM, MINGRAD = 0, 1, 2, 3


def window_averages(acc_xyz, acc_rgb, cnt):
    """Per Gaussian float32 averages over the views counted (0 where cnt = 0)."""
    cnt = np.asarray(cnt, np.int64)
    seen = cnt > 0
    ax = np.zeros(cnt.shape, np.float32)
    ar = np.zeros(cnt.shape, np.float32)
    c32 = cnt[seen].astype(np.float32)
    ax[seen] = np.asarray(acc_xyz, np.float32)[seen] / c32
    ar[seen] = np.asarray(acc_rgb, np.float32)[seen] / c32
    return ax, ar


def mingrad_scores(acc_xyz, acc_rgb, cnt, eps_xyz: float, eps_rgb: float):
    """score = max(avg_xyz / eps_xyz, avg_rgb / eps_rgb) in float32; the
    larger by a plain comparison (a NaN in the first operand yields the
    second)."""
    ax, ar = window_averages(acc_xyz, acc_rgb, cnt)
    sx = ax / np.float32(eps_xyz)
    sr = ar / np.float32(eps_rgb)
    if planted(37):
        return np.where(sx > sr, sr, sx).astype(np.float32)
    return np.where(sx > sr, sx, sr).astype(np.float32)


def select(acc_xyz, acc_rgb, cnt, frozen, eps_xyz: float, eps_rgb: float, strategy: int, fraction: float = 0.25,
           u=None):
    """New freeze map (uint8) after one update under `strategy`; the inputs
    are not modified. Returns (frozen_new, act) with act the ascending
    indices of the unfrozen Gaussians."""
    frozen = np.asarray(frozen, np.uint8)
    n = frozen.shape[0]
    cnt = np.asarray(cnt, np.int64)
    eligible = (frozen == 0) & ((cnt >= 0) if planted(38) else (cnt > 0))
    ax, ar = window_averages(acc_xyz, acc_rgb, cnt)
    new = np.zeros(n, bool)
    if strategy == RULE:
        new = eligible & (ax < np.float32(eps_xyz)) & (ar < np.float32(eps_rgb))
    elif strategy == XYZ:
        new = eligible & (ax < np.float32(eps_xyz))
    elif strategy == RANDOM:
        new = eligible & (np.asarray(u, np.float32) < np.float32(fraction))
    elif strategy == MINGRAD:
        idx = np.nonzero(eligible)[0]
        m = len(idx)
        k = int(math.floor(float(np.float32(fraction)) * m))
        if k > 0:
            score = mingrad_scores(acc_xyz, acc_rgb, cnt, eps_xyz, eps_rgb)[idx]
            order = np.lexsort((idx, score))  # by score, then index; NaN last
            new[idx[order[:k]]] = True
    else:
        raise ValueError(f"unknown strategy {strategy}")
    out = (frozen != 0) | new
    return out.astype(np.uint8), np.nonzero(~out)[0].astype(np.int32)
