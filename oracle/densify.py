"""Adaptive densification, pruning and opacity reset, written out plainly
(oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): imported by tests and
the benchmark's reference arm, never by the product path.

The paper keeps the densification of the 3DGS renderer it builds on and
changes its thresholds and cadence (Sec. 4.1): densify every 100 iterations
in [500, min(10K, early stop)), thresholds eps_den_xyz = 2e-4 and
eps_den_rgb = 1e-6 scaled over [0.5, 1.5] with the iteration like the freeze
thresholds (Eq. 5 reading), the diffuse-colour criterion used on 20% of the
densification steps, opacity reset every 3K iterations in [3K, min(10K,
early stop)], frozen Gaussians removed when they are pruned. The clone /
split / prune rules themselves are 3DGS's (not restated in the paper):

* statistics since the last densification: the average over the views in
  which the Gaussian got a gradient of |dL/dmean2d| in normalised device
  units (and of |dL/dk0|), and its largest screen radius;
* a candidate has average xyz norm >= eps_xyz (on an rgb step: or average
  rgb norm >= eps_rgb);
* a candidate whose largest scale is at most 1% of the scene extent is
  cloned (an identical copy is appended); otherwise it is split: two
  children at mean + R(q) (s * z_k), z_k ~ N(0, I_3) drawn by the caller,
  with scales s / 1.6, all else copied, and the original removed;
* then every Gaussian (originals, clones, children) with opacity < 0.005 is
  removed, and -- once past the first opacity reset -- every original whose
  largest screen radius exceeds 20 px, and every Gaussian whose largest
  scale exceeds 10% of the extent;
* output order: surviving originals in index order, then surviving clones,
  then surviving children (two per split original, child 0 first), each in
  the order of their originals; new Gaussians start unfrozen with zero Adam
  moments and statistics.

Decisions are made on the single-precision parameters with thresholds
given in the log / logit domain (log(0.01 extent), logit(0.005), ...), so
that both sides compare the same float32 numbers; child means are computed
in double precision here.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from oracle import planted


@dataclasses.dataclass
class DensifyParams:
    eps_xyz: float
    eps_rgb: float
    use_rgb: bool
    log_clone_max: float      # log(0.01 extent): largest log-scale that clones
    logit_min_opacity: float  # logit(0.005)
    prune_big: bool           # screen / world size pruning active
    max_screen_radius: int    # 20 px
    log_max_world: float      # log(0.1 extent)
    log_split_div: float      # log(1.6)
    mask_prune: bool = False  # also prune where the volume mask is off (Sec. 3.3) ...
    mask_logit_min: float = -4.595119850134589  # ... mask logit (column 59) <= logit(0.01)


def f32(x):
    return np.float32(x)


def _quat_rotation(q):
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def decisions(P, dacc_xyz, dacc_rgb, dcnt, max_radius, prm: DensifyParams) -> dict:
    """Per Gaussian: candidate, clone, split, and the prune tests of the
    original and of its copies (single-precision comparisons)."""
    P32 = np.asarray(P, np.float32)
    n = P32.shape[0]
    cnt = np.asarray(dcnt, np.int64)
    seen = cnt > 0
    avg_x = np.zeros(n, np.float32)
    avg_r = np.zeros(n, np.float32)
    avg_x[seen] = np.asarray(dacc_xyz, np.float32)[seen] / cnt[seen].astype(np.float32)
    avg_r[seen] = np.asarray(dacc_rgb, np.float32)[seen] / cnt[seen].astype(np.float32)
    cand = seen & (avg_x >= f32(prm.eps_xyz))
    if prm.use_rgb:
        cand |= seen & (avg_r >= f32(prm.eps_rgb))
    smax = P32[:, 3:6].max(axis=1) if n else np.zeros(0, np.float32)
    clone = cand & ((smax > f32(prm.log_clone_max)) if planted(27) else (smax <= f32(prm.log_clone_max)))
    split = cand & ~clone
    child_smax = (smax - f32(prm.log_split_div)).astype(np.float32)
    low_op = P32[:, 10] < f32(prm.logit_min_opacity)
    if prm.mask_prune:  # volume mask off: sigmoid(m) <= 0.01 (P carries the mask logit in column 59)
        low_op = low_op | ~(P32[:, 59] > f32(prm.mask_logit_min))
    if prm.prune_big:
        big_world = smax > f32(prm.log_max_world)
        big_child = child_smax > f32(prm.log_max_world)
        big_screen = np.asarray(max_radius, np.int64) > prm.max_screen_radius
    else:
        big_world = big_child = big_screen = np.zeros(n, bool)
    return dict(cand=cand, clone=clone, split=split, low_op=low_op, big_world=big_world, big_child=big_child,
                big_screen=big_screen)


def densify(P, dacc_xyz, dacc_rgb, dcnt, max_radius, prm: DensifyParams, z):
    """One densification and pruning step.

    P [n][59] (float32 values), statistics [n], max_radius [n] int,
    z [n_split][2][3]: the normal draws of the split Gaussians in index order.
    Returns dict(P=[n_out][59] float64, src=[n_out] source index,
    kind=[n_out] 0 original / 1 clone / 2 child 0 / 3 child 1, counts)."""
    P = np.asarray(P, np.float64)
    n = P.shape[0]
    P32 = P.astype(np.float32)
    d = decisions(P, dacc_xyz, dacc_rgb, dcnt, max_radius, prm)
    keep_orig = (True if planted(29) else ~d["split"]) & ~d["low_op"] & ~d["big_world"] & ~d["big_screen"]
    keep_clone = d["clone"] & ~d["low_op"] & ~d["big_world"]   # a clone is an exact copy, with no screen record
    keep_child = d["split"] & ~d["low_op"] & ~d["big_child"]
    split_idx = np.nonzero(d["split"])[0]
    z = np.asarray(z, np.float64).reshape(len(split_idx), 2, 3)
    rows, src, kind = [], [], []
    for i in np.nonzero(keep_orig)[0]:
        rows.append(P[i]); src.append(i); kind.append(0)
    for i in np.nonzero(keep_clone)[0]:
        rows.append(P[i]); src.append(i); kind.append(1)
    for r, i in enumerate(split_idx):
        if not keep_child[i]:
            continue
        R = _quat_rotation(P[i, 6:10])
        s = np.exp(P[i, 3:6])
        for k in range(2):
            c = P[i].copy()
            c[0:3] = P[i, 0:3] + (s * z[r, k] if planted(28) else R @ (s * z[r, k]))
            c[3:6] = [float(f32(P32[i, 3 + a] - f32(prm.log_split_div))) for a in range(3)]
            rows.append(c); src.append(i); kind.append(2 + k)
    out = np.array(rows).reshape(-1, P.shape[1]) if rows else np.zeros((0, P.shape[1]))
    counts = dict(kept=int(keep_orig.sum()), clones=int(keep_clone.sum()), children=2 * int(keep_child.sum()),
                  splits=len(split_idx))
    return dict(P=out, src=np.array(src, np.int64), kind=np.array(kind, np.int64), counts=counts)


def carry(values, src, kind, new_value=0):
    """Per-Gaussian state after densify: survivors keep theirs, new Gaussians get new_value."""
    values = np.asarray(values)
    out = np.empty((len(src),) + values.shape[1:], values.dtype)
    for k, (s, t) in enumerate(zip(src, kind)):
        out[k] = values[s] if t == 0 else new_value
    return out


def opacity_reset(P, M, V, logit_cap, frozen=None):
    """3DGS opacity reset: opacity <- min(opacity, 0.01) (here in the logit
    domain, logit_cap = logit(0.01) as float32) and the opacity's Adam moments
    set to zero, In place, for every Gaussian that is not frozen: a frozen
    Gaussian takes no parameter change until the map releases it (reading of
    Sec. 3.2.4's "no update for frozen Gaussians" for the reset of Sec. 4.1)."""
    cap = f32(logit_cap)
    sel = np.ones(P.shape[0], bool) if frozen is None else (np.asarray(frozen) == 0)
    P[sel, 10] = np.minimum(np.asarray(P[sel, 10], np.float32), cap)
    if not planted(30):
        M[sel, 10] = 0.0
        V[sel, 10] = 0.0


def opacity_to_abs(P, M, V, rescale: bool = False):
    """Start of the finetuning stage's absolute-value opacity (Sec. 4.1): the
    opacity parameter x becomes o = sigmoid(x), so |new x| is the same
    opacity. Its Adam moments either restart at zero or (rescale) are carried
    over: the new parameter's gradient is the old one over s = o (1 - o), so
    m / s and v / s^2 (s floored at 1e-12). In place."""
    x = np.asarray(P[:, 10], np.float64)
    o = 1.0 / (1.0 + np.exp(-x))
    P[:, 10] = o
    if rescale:
        s = np.maximum(o * (1.0 - o), 1e-12)
        M[:, 10] = M[:, 10] / s
        V[:, 10] = V[:, 10] / (s * s)
    else:
        M[:, 10] = 0.0
        V[:, 10] = 0.0


def logit(p: float) -> float:
    return math.log(p / (1.0 - p))
