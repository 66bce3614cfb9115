"""Central finite differences of the FP64 oracle's Eq. 3 loss for single
parameters of a large scene, computed locally (a helper of the 3M-Gaussian
test; it runs in spawned worker processes).

The loss is taken on a crop of the image. Moving one parameter of Gaussian i
changes only the pixels of the tiles of its rectangle (before and after the
move), so the change of the crop's loss equals the change of the share
(oracle.loss_window) of the window W1 = those pixels widened by the SSIM
radius (5), and that share reads the image only inside W2 = W1 widened by 5
more. Each evaluation therefore re-projects Gaussian i alone, re-sorts only
the Gaussians whose rectangles meet W2 (in their original order, which keeps
the depth tie-break), renders the pixels of W2 and evaluates the window share.
"""
from __future__ import annotations

import numpy as np

import oracle

_S: dict = {}


def init(state: dict):
    """Worker state: P (n, 59) float64, proj (oracle projection of P), cam
    (synth.Camera, already float32-rounded), tile, crop (x0, y0, size), gt
    (3, size, size)."""
    _S.update(state)
    _S["ocam"] = oracle.make_cam(state["cam"], tile=state["tile"])


def _tile_box_to_pixels(r, tile, crop):
    x0, y0, cs = crop
    px0, py0, px1, py1 = r[0] * tile, r[1] * tile, r[2] * tile, r[3] * tile
    return max(px0, x0), max(py0, y0), min(px1, x0 + cs), min(py1, y0 + cs)


def local_fd(task):
    """task = (i, j, hs[, locked]): Gaussian i (row of P), parameter j, steps
    hs. Returns [(L(+h) - L(-h)) / 2h for h in hs]. locked: the renders keep
    the tile lists and every per-pixel decision (skip, alpha cap, stop) of
    the unperturbed point (oracle.render_pixels_locked), so the difference
    quotient approaches the derivative of the smooth piece the point lies on
    -- the derivative the analytic backward computes -- even where a step of
    h would move a decision."""
    if len(task) == 4 and task[3]:
        return _local_fd_locked(*task[:3])
    i, j, hs = task[:3]
    P, proj, ocam, tile, crop, gt = _S["P"], _S["proj"], _S["ocam"], _S["tile"], _S["crop"], _S["gt"]
    x0, y0, cs = crop
    rows = []
    for h in hs:
        for sgn in (1.0, -1.0):
            r = P[i].copy()
            r[j] += sgn * h
            rows.append(r)
    pert = oracle.project(np.array(rows), ocam)
    rects = np.vstack([proj["rect"][i:i + 1], pert["rect"][pert["radius"] > 0]])
    box = (rects[:, 0].min(), rects[:, 1].min(), rects[:, 2].max(), rects[:, 3].max())
    bx0, by0, bx1, by1 = _tile_box_to_pixels(box, tile, crop)
    if bx0 >= bx1 or by0 >= by1:
        return [0.0 for _ in hs]
    w1 = (max(bx0 - 5, x0), max(by0 - 5, y0), min(bx1 + 5, x0 + cs), min(by1 + 5, y0 + cs))
    w2 = (max(w1[0] - 5, x0), max(w1[1] - 5, y0), min(w1[2] + 5, x0 + cs), min(w1[3] + 5, y0 + cs))
    # Gaussians whose rectangle meets the tiles of W2, in their original order
    t0x, t0y, t1x, t1y = w2[0] // tile, w2[1] // tile, (w2[2] - 1) // tile + 1, (w2[3] - 1) // tile + 1
    R = proj["rect"]
    sub = np.nonzero((proj["radius"] > 0) & (R[:, 0] < t1x) & (R[:, 2] > t0x) & (R[:, 1] < t1y) & (R[:, 3] > t0y))[0]
    if not np.any(sub == i):
        sub = np.sort(np.append(sub, i))
    k = int(np.nonzero(sub == i)[0][0])
    base = {key: proj[key][sub].copy() for key in ("mean2d", "conic", "depth", "opacity", "rgb", "radius", "rect")}
    yy, xx = np.meshgrid(np.arange(w2[1], w2[3]), np.arange(w2[0], w2[2]), indexing="ij")
    px, py = xx.ravel(), yy.ravel()
    out = []
    for q, h in enumerate(hs):
        L = []
        for s in range(2):
            row = 2 * q + s
            pr = {key: v.copy() for key, v in base.items()}
            for key in pr:
                pr[key][k] = pert[key][row]
            vals, ranges = oracle.sort_proj(pr, ocam.width, ocam.height, tile)
            ren = oracle.render_pixels(pr, vals, ranges, ocam, px, py)
            img = np.zeros((3, cs, cs))
            img[:, py - y0, px - x0] = ren["image"]
            L.append(oracle.loss_window(img, gt, w1[0] - x0, w1[1] - y0, w1[2] - x0, w1[3] - y0))
        out.append((L[0] - L[1]) / (2 * h))
    return out


def _local_fd_locked(i, j, hs):
    P, proj, ocam, tile, crop, gt = _S["P"], _S["proj"], _S["ocam"], _S["tile"], _S["crop"], _S["gt"]
    x0, y0, cs = crop
    if proj["radius"][i] <= 0:
        return [0.0 for _ in hs]
    bx0, by0, bx1, by1 = _tile_box_to_pixels(proj["rect"][i], tile, crop)
    if bx0 >= bx1 or by0 >= by1:
        return [0.0 for _ in hs]
    w1 = (max(bx0 - 5, x0), max(by0 - 5, y0), min(bx1 + 5, x0 + cs), min(by1 + 5, y0 + cs))
    w2 = (max(w1[0] - 5, x0), max(w1[1] - 5, y0), min(w1[2] + 5, x0 + cs), min(w1[3] + 5, y0 + cs))
    t0x, t0y, t1x, t1y = w2[0] // tile, w2[1] // tile, (w2[2] - 1) // tile + 1, (w2[3] - 1) // tile + 1
    R = proj["rect"]
    sub = np.nonzero((proj["radius"] > 0) & (R[:, 0] < t1x) & (R[:, 2] > t0x) & (R[:, 1] < t1y) & (R[:, 3] > t0y))[0]
    k = int(np.nonzero(sub == i)[0][0])
    base = {key: proj[key][sub].copy() for key in ("mean2d", "conic", "depth", "opacity", "rgb", "radius")}
    vals, ranges = oracle.sort_proj(base, ocam.width, ocam.height, tile)
    yy, xx = np.meshgrid(np.arange(w2[1], w2[3]), np.arange(w2[0], w2[2]), indexing="ij")
    px, py = xx.ravel(), yy.ravel()
    _, dec = oracle.render_pixels_locked(base, vals, ranges, ocam, px, py)
    rows = []
    for h in hs:
        for sgn in (1.0, -1.0):
            r = P[i].copy()
            r[j] += sgn * h
            rows.append(r)
    pert = oracle.project(np.array(rows), ocam)
    out = []
    for q, h in enumerate(hs):
        L = []
        for s in range(2):
            pr = {key: v.copy() for key, v in base.items()}
            for key in ("mean2d", "conic", "opacity", "rgb"):
                pr[key][k] = pert[key][2 * q + s]
            image, _ = oracle.render_pixels_locked(pr, vals, ranges, ocam, px, py, dec)
            img = np.zeros((3, cs, cs))
            img[:, py - y0, px - x0] = image
            L.append(oracle.loss_window(img, gt, w1[0] - x0, w1[1] - y0, w1[2] - x0, w1[3] - y0))
        out.append((L[0] - L[1]) / (2 * h))
    return out
