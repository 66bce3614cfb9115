"""Helpers for the GPU-vs-oracle parity tests.

Inputs are rounded to float32 once; the CUDA path receives the float32 values
and the FP64 oracle receives the same values widened to float64, so the two
sides differ only by the arithmetic each performs.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2504_06716_gb300 import lib, synth

# A decision (alpha floor/cap, transmittance floor, exponent sign) whose
# oracle value lies within this relative distance of its threshold may go
# either way in float32; such pixels are compared for validity only.
PIXEL_MARGIN = 1e-5
# Same for the integer decisions of the projection (radius, tile rectangle,
# near plane), in pixels / world units.
PROJ_MARGIN = 1e-3
# When the CUDA path also computes the projection itself, its alpha values
# differ from the oracle's by up to ~5e-5 relative (float32 2-D means and
# conics); decisions within this margin may go either way.
E2E_PIXEL_MARGIN = 2e-4

GRAD2D_KEYS = [("d_mean2d", 0), ("d_mean2d", 1), ("d_conic", 0), ("d_conic", 1), ("d_conic", 2), ("d_opacity", None),
               ("d_rgb", 0), ("d_rgb", 1), ("d_rgb", 2)]


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def round_camera(cam: synth.Camera) -> synth.Camera:
    return synth.Camera(cam.width, cam.height, float(np.float32(cam.fx)), float(np.float32(cam.fy)),
                        float(np.float32(cam.cx)), float(np.float32(cam.cy)), f32(cam.R), f32(cam.t), f32(cam.campos))


def cameras(cam: synth.Camera, tile=16, bg=(0.0, 0.0, 0.0), dilation=0.3, znear=0.2):
    """(oracle camera, GPU camera) describing the same float32 camera."""
    c = round_camera(cam)
    bg = tuple(float(v) for v in f32(bg))
    return (oracle.make_cam(c, tile=tile, bg=bg, dilation=float(np.float32(dilation)), znear=float(np.float32(znear))),
            lib.camera(c, tile=tile, bg=bg, dilation=dilation, znear=znear))


def records_from_oracle(proj: dict) -> np.ndarray:
    """Oracle projection -> float32 splat records [n][12] (the C-ABI layout)."""
    n = proj["radius"].shape[0]
    rec = np.zeros((n, 12), np.float32)
    rec[:, 0:2] = proj["mean2d"]
    rec[:, 2:5] = proj["conic"]
    rec[:, 5] = proj["opacity"]
    rec[:, 6:9] = proj["rgb"]
    rec[:, 9] = proj["depth"]
    rec[:, 10] = proj["radius"].astype(np.int32).view(np.float32)
    rec[:, 11] = proj["tiles_touched"].astype(np.int32).view(np.float32)
    return rec


def proj_from_records(rec: np.ndarray) -> dict:
    """float32 splat records -> the oracle's per-Gaussian arrays (float64 copies of the same values)."""
    return dict(mean2d=rec[:, 0:2].astype(np.float64), conic=rec[:, 2:5].astype(np.float64),
                opacity=rec[:, 5].astype(np.float64), rgb=rec[:, 6:9].astype(np.float64),
                depth=rec[:, 9].astype(np.float64), radius=rec[:, 10].view(np.int32).copy(),
                tiles_touched=rec[:, 11].view(np.int32).copy())


def pack64(p59: np.ndarray) -> np.ndarray:
    out = np.zeros((p59.shape[0], 64), np.float32)
    out[:, :59] = p59
    return out


def close(got, want, rtol, floor, mask=None):
    """Elementwise |got - want| <= rtol * (|want| + floor); returns (ok, worst ratio)."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    err = np.abs(got - want)
    lim = rtol * (np.abs(want) + floor)
    if mask is not None:
        err = err[mask]
        lim = lim[mask]
    if err.size == 0:
        return True, 0.0
    ratio = float((err / np.maximum(lim, 1e-300)).max())
    return ratio <= 1.0, ratio


def grad2d_matrix(bwd: dict) -> np.ndarray:
    """Oracle raster gradients as an [n][9] array in the grad2d column order."""
    n = bwd["d_opacity"].shape[0]
    out = np.zeros((n, 9))
    for k, (key, col) in enumerate(GRAD2D_KEYS):
        out[:, k] = bwd[key] if col is None else bwd[key][:, col]
    return out


def param_bound(P, ocam, amb_abs, frozen=None, sh_degree=3):
    """Bound on |change of the 59-parameter gradient| caused by raster-gradient
    changes of at most amb_abs[n][9]: sum_k |J[:, k]| amb_abs[k], with the
    columns of the (per-Gaussian) projection Jacobian J obtained from the
    oracle's projection backward on unit raster gradients."""
    n = P.shape[0]
    bound = np.zeros((n, 59))
    if not np.any(amb_abs):
        return bound
    for k, (key, col) in enumerate(GRAD2D_KEYS):
        g2 = dict(d_mean2d=np.zeros((n, 2)), d_conic=np.zeros((n, 3)), d_opacity=np.zeros(n), d_rgb=np.zeros((n, 3)))
        if col is None:
            g2[key][:] = 1.0
        else:
            g2[key][:, col] = 1.0
        Jk = oracle.project_bwd(P, ocam, g2, frozen, sh_degree)["G"]
        bound += np.abs(Jk) * amb_abs[:, k:k + 1]
    return bound


def close_bound(got, want, rtol, floor, extra, mask=None):
    """|got - want| <= rtol * (|want| + floor) + extra; returns (ok, worst ratio)."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    err = np.abs(got - want)
    lim = rtol * (np.abs(want) + floor) + extra
    if mask is not None:
        err, lim = err[mask], lim[mask]
    if err.size == 0:
        return True, 0.0
    ratio = float((err / np.maximum(lim, 1e-300)).max())
    return ratio <= 1.0, ratio


# The CUDA sort lists a splat in a tile when the box of the tile's pixel
# centres holds a point with q = d^T Q d <= tau + 1e-3 (1 + tau), tau =
# 2 ln(255 o), tested in float32; the oracle lists it when a pixel centre of
# the tile inside the image has alpha >= 1/255, in double precision. So the
# CUDA lists hold the oracle's, and every further entry lies within this
# band of the floor (box minimum of q in double precision).
LIST_BAND = 2e-3


def box_min_q(mx, my, a, b, c, X0, Y0, X1, Y1):
    """Least value of q = a dx^2 + 2 b dx dy + c dy^2 (d = point - mean) over
    the boxes [X0, X1] x [Y0, Y1], in double precision: 0 when the mean lies
    inside, else the least of the four edges' clamped one-dimensional minima
    (q is convex, so its minimum over a box without the mean is on the edge)."""
    inside = (mx >= X0) & (mx <= X1) & (my >= Y0) & (my <= Y1)
    best = np.full(np.shape(mx), np.inf)
    for ex in (X0, X1):
        dx = ex - mx
        dy = np.clip(-(b / c) * dx, Y0 - my, Y1 - my)
        best = np.minimum(best, a * dx * dx + 2 * b * dx * dy + c * dy * dy)
    for ey in (Y0, Y1):
        dy = ey - my
        dx = np.clip(-(b / a) * dy, X0 - mx, X1 - mx)
        best = np.minimum(best, a * dx * dx + 2 * b * dx * dy + c * dy * dy)
    return np.where(inside, 0.0, best)


def _entries(vals, ranges):
    """(tile, splat) of every entry, checking that the ranges tile the list in order."""
    ranges = np.asarray(ranges, np.int64).reshape(-1, 2)
    cnt = ranges[:, 1] - ranges[:, 0]
    assert np.all(cnt >= 0)
    ne = np.nonzero(cnt)[0]
    if ne.size:
        assert ranges[ne[0], 0] == 0 and np.all(ranges[ne[1:], 0] == ranges[ne[:-1], 1])
    tiles = np.repeat(np.arange(ranges.shape[0], dtype=np.int64), cnt)
    return tiles, np.asarray(vals, np.int64)[: tiles.size] & 0xFFFFFFFF


def check_lists(vals, ranges, want_vals, want_ranges, rec, tile: int, tiles_x: int) -> int:
    """The CUDA tile lists against the oracle's: every oracle entry present, in
    the same order; every CUDA-only entry within LIST_BAND of the alpha floor;
    each tile's list in ascending (float32 depth, index). Returns the number of
    CUDA-only entries."""
    gt, gs = _entries(vals, ranges)
    wt, ws = _entries(want_vals, want_ranges)
    gkey, wkey = (gt << 32) | gs, (wt << 32) | ws
    member = np.isin(gkey, wkey)
    assert np.array_equal(gkey[member], wkey), "oracle entries missing or out of order"
    dbits = np.ascontiguousarray(rec[:, 9], np.float32).view(np.uint32).astype(np.int64)
    order = np.stack([gt, dbits[gs], gs], 1)
    same = gt[1:] == gt[:-1]
    step = order[1:] - order[:-1]
    first = np.where(step[:, 1] != 0, step[:, 1], step[:, 2])
    assert np.all(first[same] > 0), "a tile's list is not in (depth, index) order"
    xt, xs = gt[~member], gs[~member]
    if xt.size:
        r = rec[xs].astype(np.float64)
        X0, Y0 = (xt % tiles_x) * tile, (xt // tiles_x) * tile
        q = box_min_q(r[:, 0], r[:, 1], r[:, 2], r[:, 3], r[:, 4], X0, Y0, X0 + tile - 1, Y0 + tile - 1)
        tau = 2 * np.log(np.maximum(255.0 * r[:, 5], 1e-300))
        assert np.all(255.0 * r[:, 5] >= 1.0 - 1e-6)
        worst = float(np.max(q - tau - LIST_BAND * (1 + np.abs(tau))))
        assert worst <= 0.0, f"a CUDA-only entry lies outside the band (excess {worst:.3e})"
    return int(xt.size)


# The L1 term of Eq. 3 takes the sign of image - target: where the two agree
# to within this margin, float32 and double may take different signs, and
# dL/dC of that channel then differs by 2 (1 - lambda) / (3 H W).
L1_MARGIN = 1e-5


def l1_sign_bound(proj, vals, ranges, ocam, image, gt, frozen=None, lam=0.2):
    """Bound [n][9] on the raster-gradient change that an L1 sign taken the
    other way may cause: the oracle's raster backward with dL/dC set to the
    largest change at the ambiguous channels and 0 elsewhere, its terms taken
    in absolute value. Pixels where image and target are both exactly zero
    decide alike on both sides (sign 0)."""
    amb = np.abs(image - gt) <= L1_MARGIN
    amb &= ~((image == 0) & (gt == 0))
    dl = np.where(amb, 2.0 * (1.0 - lam) / image.size, 0.0)
    rb = oracle.render_bwd(proj, vals, ranges, ocam, dl, frozen, amb.any(axis=0).astype(np.uint8))
    return rb["amb_abs"]
