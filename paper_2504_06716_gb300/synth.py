"""Seeded synthetic inputs: Gaussian sets and pinhole cameras.

This module draws inputs only. It holds none of the method's arithmetic (no
projection, colour, compositing, loss or optimiser maths), so both the CUDA
path and the FP64 oracle may consume what it produces.

The paper trains on Mip-NeRF 360, Tanks&Temples and Deep Blending scenes with
SfM initialisation (Sec. 4.1); none of that data is available here, so these
seeded scenes stand in for them:

* ``tiny_scene`` -- 2,000 Gaussians in the cube [-1, 1]^3, a 3,000-Gaussian
  ground-truth set, eight 128x128 cameras on a radius-4 circle.
* ``surface_scene`` -- Gaussians sampled on a unit sphere, a ground plane and
  20 boxes, cameras on a hemisphere (1M/1.5M Gaussians at 1237x822 for the
  mid-size workload, 3M at 1920x1080 for the stress workload).

Parameter order of the (N, 59) arrays returned here, one row per Gaussian:
  0-2   mean (x, y, z) in world units
  3-5   log of the three axis scales
  6-9   rotation quaternion (w, x, y, z), not normalised
  10    opacity logit
  11-58 spherical-harmonic coefficients, coefficient-major: 11 + 3*c + ch for
        coefficient c = 0..15 and colour channel ch = 0..2
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

N_PARAMS = 59
N_SH = 16


@dataclasses.dataclass
class Camera:
    """A pinhole camera. ``R``/``t`` map world points into camera space
    (x right, y down, z forward): p_cam = R @ p_world + t."""

    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray  # (3, 3) float64
    t: np.ndarray  # (3,) float64
    campos: np.ndarray  # (3,) float64, camera centre in world space


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def look_at(eye, target, up) -> tuple[np.ndarray, np.ndarray]:
    """Rotation and translation of a camera at ``eye`` looking at ``target``."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ eye
    return R, t


def pinhole(width: int, height: int, fov_x_deg: float, eye, target=(0, 0, 0), up=(0, 0, 1)) -> Camera:
    fx = width / (2.0 * math.tan(math.radians(fov_x_deg) / 2.0))
    R, t = look_at(eye, target, up)
    return Camera(width, height, fx, fx, width / 2.0, height / 2.0, R, t, np.asarray(eye, np.float64))


def circle_cameras(n: int, radius: float, width: int, height: int, fov_x_deg: float = 60.0) -> list[Camera]:
    """``n`` cameras evenly spaced on a circle of ``radius`` in the z = 0 plane, looking at the origin."""
    cams = []
    for i in range(n):
        a = 2.0 * math.pi * i / n
        cams.append(pinhole(width, height, fov_x_deg, (radius * math.cos(a), radius * math.sin(a), 0.0)))
    return cams


def hemisphere_cameras(n: int, radius: float, width: int, height: int, fov_x_deg: float = 60.0) -> list[Camera]:
    """``n`` cameras on a Fibonacci spiral over the upper (y > 0) hemisphere, looking at the origin."""
    golden = math.pi * (3.0 - math.sqrt(5.0))
    cams = []
    for i in range(n):
        y = 0.15 + 0.8 * (i + 0.5) / n
        r = math.sqrt(1.0 - y * y)
        a = golden * i
        eye = (radius * r * math.cos(a), radius * y, radius * r * math.sin(a))
        cams.append(pinhole(width, height, fov_x_deg, eye, up=(0, 1, 0)))
    return cams


def _random_quats(g: np.random.Generator, n: int) -> np.ndarray:
    q = g.standard_normal((n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def gaussians_uniform(n: int, seed: int) -> np.ndarray:
    """(n, 59) float64: means U[-1,1]^3, log-scales N(-3.5, 0.3), random unit
    quaternions, opacity logits U(-2, 2), SH DC coefficients U(0, 1) and
    higher-band coefficients N(0, 0.05)."""
    g = _rng(seed)
    p = np.zeros((n, N_PARAMS), np.float64)
    p[:, 0:3] = g.uniform(-1.0, 1.0, (n, 3))
    p[:, 3:6] = g.normal(-3.5, 0.3, (n, 3))
    p[:, 6:10] = _random_quats(g, n)
    p[:, 10] = g.uniform(-2.0, 2.0, n)
    sh = g.normal(0.0, 0.05, (n, N_SH, 3))
    sh[:, 0, :] = g.uniform(0.0, 1.0, (n, 3))
    p[:, 11:] = sh.reshape(n, 48)
    return p


def _sample_surfaces(g: np.random.Generator, n: int, n_boxes: int = 20):
    """Points and unit normals on a mix of a unit sphere, the plane y = -1.2
    over [-4, 4]^2 and ``n_boxes`` axis-aligned boxes standing on it, drawn
    with probability proportional to area. The box layout depends on the
    generator state only, so two calls with the same seed share it."""
    box_g = _rng(12345)  # box layout is fixed for every scene drawn here
    centres = box_g.uniform(-3.0, 3.0, (n_boxes, 2))
    sizes = box_g.uniform(0.1, 0.6, (n_boxes, 3))
    faces = []  # (area, origin, edge u, edge v, normal)
    faces.append((64.0, np.array([-4.0, -1.2, -4.0]), np.array([8.0, 0, 0]), np.array([0, 0, 8.0]), np.array([0, 1.0, 0])))
    for (cx, cz), (sx, sy, sz) in zip(centres, sizes):
        x0, x1 = cx - sx / 2, cx + sx / 2
        z0, z1 = cz - sz / 2, cz + sz / 2
        y0, y1 = -1.2, -1.2 + sy
        faces += [
            (sx * sz, np.array([x0, y1, z0]), np.array([sx, 0, 0]), np.array([0, 0, sz]), np.array([0, 1.0, 0])),
            (sx * sy, np.array([x0, y0, z0]), np.array([sx, 0, 0]), np.array([0, sy, 0]), np.array([0, 0, -1.0])),
            (sx * sy, np.array([x0, y0, z1]), np.array([sx, 0, 0]), np.array([0, sy, 0]), np.array([0, 0, 1.0])),
            (sz * sy, np.array([x0, y0, z0]), np.array([0, 0, sz]), np.array([0, sy, 0]), np.array([-1.0, 0, 0])),
            (sz * sy, np.array([x1, y0, z0]), np.array([0, 0, sz]), np.array([0, sy, 0]), np.array([1.0, 0, 0])),
        ]
    sphere_area = 4.0 * math.pi
    areas = np.array([sphere_area] + [f[0] for f in faces])
    which = g.choice(len(areas), size=n, p=areas / areas.sum())
    pts = np.empty((n, 3))
    nrm = np.empty((n, 3))
    on_sphere = which == 0
    k = int(on_sphere.sum())
    v = g.standard_normal((k, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    pts[on_sphere] = v
    nrm[on_sphere] = v
    for fi, (_, o, eu, ev, fn) in enumerate(faces, start=1):
        sel = which == fi
        m = int(sel.sum())
        if m == 0:
            continue
        uv = g.uniform(0.0, 1.0, (m, 2))
        pts[sel] = o + uv[:, :1] * eu + uv[:, 1:] * ev
        nrm[sel] = fn
    return pts, nrm


def gaussians_surface(n: int, seed: int, ground_truth: bool = False) -> np.ndarray:
    """(n, 59) float64 Gaussians on the sphere/plane/box surface mix, with
    N(0, 0.01) positional jitter and log-scales N(-4.5, 0.5).

    ``ground_truth=True`` gives the target set: opaque (logits U(2, 4)), DC
    colour coefficients = low-frequency sinusoids of position plus per-Gaussian
    texture noise N(0, 0.3), and view-dependent higher bands N(0, 0.03). The
    training Gaussians sit elsewhere on the same surfaces and cannot reproduce
    the texture exactly, so the fit saturates as on captured scenes instead of
    converging to the target. Otherwise the training initialisation: logits
    U(-2, 2), DC coefficients U(0, 1), higher bands N(0, 0.05)."""
    g = _rng(seed)
    pts, _ = _sample_surfaces(g, n)
    p = np.zeros((n, N_PARAMS), np.float64)
    p[:, 0:3] = pts + g.normal(0.0, 0.01, (n, 3))
    p[:, 3:6] = g.normal(-4.5, 0.5, (n, 3))
    p[:, 6:10] = _random_quats(g, n)
    if ground_truth:
        p[:, 10] = g.uniform(2.0, 4.0, n)
        x, y, z = p[:, 0], p[:, 1], p[:, 2]
        p[:, 11] = 0.6 * np.sin(1.7 * x + 0.3) + 0.4 * np.cos(2.3 * z)
        p[:, 12] = 0.6 * np.sin(2.1 * z - 0.7) + 0.4 * np.cos(1.3 * y + x)
        p[:, 13] = 0.6 * np.cos(1.1 * x - 1.9 * z) + 0.3 * np.sin(3.1 * y)
        p[:, 11:14] += g.normal(0.0, 0.3, (n, 3))
        p[:, 14:] = g.normal(0.0, 0.03, (n, 45))
    else:
        p[:, 10] = g.uniform(-2.0, 2.0, n)
        sh = g.normal(0.0, 0.05, (n, N_SH, 3))
        sh[:, 0, :] = g.uniform(0.0, 1.0, (n, 3))
        p[:, 11:] = sh.reshape(n, 48)
    return p


@dataclasses.dataclass
class Scene:
    init: np.ndarray  # (N, 59) training initialisation
    gt: np.ndarray  # (M, 59) ground-truth Gaussians the targets are rendered from
    cameras: list[Camera]
    train_views: list[int]
    test_views: list[int]
    subset_views: list[int]  # training views used for the early-stop PSNR


def split_views(n_views: int, subset_frac: float, seed: int):
    """Every 8th view is held out for testing (Sec. 4.1); a seeded
    ``subset_frac`` of the training views forms the early-stop subset."""
    test = [i for i in range(n_views) if i % 8 == 7]
    train = [i for i in range(n_views) if i % 8 != 7]
    k = max(1, int(round(subset_frac * len(train))))
    subset = sorted(_rng(seed).choice(train, size=k, replace=False).tolist())
    return train, test, subset


def tiny_scene(seed: int = 0) -> Scene:
    """2,000 training Gaussians, 3,000 ground-truth Gaussians, 8 cameras at 128x128
    (seed 0: initialisation seed 0, ground-truth seed 1)."""
    cams = circle_cameras(8, 4.0, 128, 128, 60.0)
    train, test, subset = split_views(8, 0.1, 2)
    return Scene(gaussians_uniform(2000, 2 * seed), gaussians_uniform(3000, 2 * seed + 1), cams, train, test, subset)


def surface_scene(n_init: int, n_gt: int, n_views: int, width: int, height: int, seed: int = 0) -> Scene:
    cams = hemisphere_cameras(n_views, 4.0, width, height, 60.0)
    train, test, subset = split_views(n_views, 0.1, seed + 2)
    return Scene(
        gaussians_surface(n_init, seed, ground_truth=False),
        gaussians_surface(n_gt, seed + 1, ground_truth=True),
        cams,
        train,
        test,
        subset,
    )


def smooth_image(height: int, width: int, seed: int, terms: int = 6) -> np.ndarray:
    """(3, height, width) float64 target image in [0, 1]: per channel a sum of
    ``terms`` random plane waves (wavelengths 8 to 128 pixels), rescaled."""
    g = _rng(seed)
    yy, xx = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    out = np.zeros((3, height, width))
    for c in range(3):
        for _ in range(terms):
            k = 2 * math.pi / g.uniform(8.0, 128.0)
            a = g.uniform(0.0, 2 * math.pi)
            out[c] += g.uniform(0.2, 1.0) * np.sin(k * (math.cos(a) * xx + math.sin(a) * yy) + g.uniform(0, 2 * math.pi))
        lo, hi = out[c].min(), out[c].max()
        out[c] = (out[c] - lo) / max(hi - lo, 1e-12)
    return out


def view_order(n_iters: int, train_views: list[int], seed: int) -> list[int]:
    """Training view per iteration: a fresh seeded permutation of the training views each epoch."""
    g = _rng(seed)
    out: list[int] = []
    while len(out) < n_iters:
        out += [train_views[i] for i in g.permutation(len(train_views))]
    return out[:n_iters]
