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
