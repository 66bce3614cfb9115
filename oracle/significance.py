"""Significance pruning (Sec. 3.3 "Pruning with Significance of Gaussians",
after LightGaussian; Sec. 4.1: at 4K and 7K, removal 75% with decay 0.8),
written out plainly (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): imported by tests and
the benchmark's reference arm, never by the product path.

Readings (the paper names the method and its schedule only):

* hits_i: over the training views, the number of pixels whose colour blends
  Gaussian i (its entries before the pixel's stop with alpha >= 1/255 and a
  non-positive exponent: the contributors of Eq. 2);
* score_i = hits_i * o_i * (V_i / V_q)^beta, V_i = exp(s_0 + s_1 + s_2) the
  product of the scales, V_q the volume of rank floor(q n) - 1 in ascending
  (volume, index) order, q = 0.9, beta = 0.1 (LightGaussian's volume power);
* the floor(f n) Gaussians of lowest (score, index) are removed, f = 0.75 at
  the first pruning and 0.75 * 0.8 at the second.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

QUANTILE, BETA, FRACTION, DECAY = 0.9, 0.1, 0.75, 0.8


def hit_counts(proj: dict, vals, ranges, cam, n: int) -> np.ndarray:
    """Per Gaussian, the pixels of one view that blend it (oracle render decisions)."""
    hits = np.zeros(n, np.int64)
    for py in range(cam.height):
        for px in range(cam.width):
            pos, _, _ = oracle.pixel_trace(proj, vals, ranges, cam, px, py)
            t = (py // cam.tile) * ((cam.width + cam.tile - 1) // cam.tile) + px // cam.tile
            for p in pos:
                hits[vals[ranges[t][0] + p]] += 1
    return hits


def scores(P, hits, beta: float = BETA, quantile: float = QUANTILE, opacity_abs: bool = False) -> np.ndarray:
    P = np.asarray(P, np.float64)
    n = P.shape[0]
    vol = np.exp(P[:, 3] + P[:, 4] + P[:, 5])
    order = np.lexsort((np.arange(n), vol))
    k = int(math.floor(quantile * n))
    v_q = vol[order[k - 1]] if k >= 1 else 0.0
    o = np.abs(P[:, 10]) if opacity_abs else 1.0 / (1.0 + np.exp(-P[:, 10]))
    if oracle.planted(34):
        o = 1.0
    v = (vol / v_q) ** beta if v_q > 0 else np.ones(n)
    return np.asarray(hits, np.float64) * o * v


def mark(score, fraction: float) -> np.ndarray:
    """1 for the floor(fraction n) lowest (score, index), else 0."""
    score = np.asarray(score, np.float64)
    n = score.shape[0]
    k = int(math.floor(fraction * n))
    out = np.zeros(n, np.uint8)
    if k > 0:
        order = np.lexsort((np.arange(n), score))
        out[(order[::-1] if oracle.planted(35) else order)[:k]] = 1
    return out
