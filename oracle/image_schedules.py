"""Image-space schedules of the Trick-GS additions (Sec. 3.3 "Progressive
Training" and "Blur"; Sec. 4.1), written out plainly (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): imported by tests and
the benchmark's reference arm, never by the product path.

The paper trains on lower-resolution images first and raises the resolution
with a cosine schedule until iteration 6K, starting at scale 0.175; it also
blurs the training images with a Gaussian whose size decays until 6K
(Sec. 3.3 says a cosine schedule, Sec. 4.1 a log one; the kernel starts at
5x5). Readings taken here:

* scale s(k) = s0 + (1 - s0) (1 - cos(pi min(k, K) / K)) / 2, s0 = 0.175,
  K = 6000; the image is W_k x H_k = max(1, round(s W)) x max(1, round(s H))
  covering the same extent of the image plane: with pixel j spanning
  [j - 1/2, j + 1/2), the plane [-1/2, W - 1/2) maps onto [-1/2, W_k - 1/2),
  u' = (u + 1/2) r - 1/2 with r = W_k / W (r_y = H_k / H for v), so the
  camera becomes fx' = r fx, cx' = (cx + 1/2) r - 1/2 (same for y);
* the target at that size is the area average of the full-resolution
  target: target pixel i covers the source interval [i / r - 1/2,
  (i + 1) / r - 1/2), each source pixel weighted by its overlap (rows sum to
  one; the intervals tile the image exactly), separable in x and y;
* blur: a Gaussian of standard deviation sigma(k) = sigma0 (1 + cos(pi
  min(k, K) / K)) / 2 pixels of the current image (the cosine of Sec. 3.3),
  sigma0 = 1, on a 5 x 5 window, its weights normalised over the taps that
  fall inside the image; no blur once sigma < 0.1.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import planted

S0, K_PROG, SIGMA0, K_BLUR, SIGMA_MIN, BLUR_RADIUS = 0.175, 6000, 1.0, 6000, 0.1, 2


def scale_at(k: int, s0: float = S0, K: int = K_PROG) -> float:
    t = min(k, K) / K
    return s0 + (1.0 - s0) * (1.0 - math.cos(math.pi * t)) / 2.0


def size_at(k: int, W: int, H: int, s0: float = S0, K: int = K_PROG) -> tuple[int, int]:
    s = scale_at(k, s0, K)
    return max(1, int(round(s * W))), max(1, int(round(s * H)))


def sigma_at(k: int, sigma0: float = SIGMA0, K: int = K_BLUR) -> float:
    t = min(k, K) / K
    return sigma0 * (1.0 + math.cos(math.pi * t)) / 2.0


def area_weights(n_src: int, n_dst: int) -> np.ndarray:
    """[n_dst][n_src] weights of the 1-D area average (rows sum to 1)."""
    r = n_dst / n_src
    Wm = np.zeros((n_dst, n_src))
    for i in range(n_dst):
        a, b = (i / r, (i + 1) / r) if planted(40) else (i / r - 0.5, (i + 1) / r - 0.5)
        for j in range(n_src):
            ov = min(b, j + 0.5) - max(a, j - 0.5)
            if ov > 0:
                Wm[i, j] = ov
        Wm[i] /= Wm[i].sum()
    return Wm


def resize_area(img, W2: int, H2: int) -> np.ndarray:
    """[C][H][W] -> [C][H2][W2] area average (float64)."""
    img = np.asarray(img, np.float64)
    _, H, W = img.shape
    Ax, Ay = area_weights(W, W2), area_weights(H, H2)
    return np.stack([Ay @ img[c] @ Ax.T for c in range(img.shape[0])])


def camera_at(fx: float, fy: float, cx: float, cy: float, W: int, H: int, W2: int, H2: int):
    """Intrinsics of the W2 x H2 image covering the same extent of the image plane."""
    rx, ry = W2 / W, H2 / H
    if planted(39):
        return fx * rx, fy * ry, cx * rx, cy * ry
    return fx * rx, fy * ry, (cx + 0.5) * rx - 0.5, (cy + 0.5) * ry - 0.5


def blur(img, sigma: float, radius: int = BLUR_RADIUS) -> np.ndarray:
    """[C][H][W] Gaussian blur, weights renormalised over in-image taps; the
    input itself when sigma < SIGMA_MIN."""
    img = np.asarray(img, np.float64)
    if sigma < SIGMA_MIN:
        return img.copy()
    C, H, W = img.shape
    out = np.zeros_like(img)
    for y in range(H):
        for x in range(W):
            acc = np.zeros(C)
            wsum = 0.0
            for dy in range(-radius, radius + 1):
                for dx in range(-radius, radius + 1):
                    yy, xx = y + dy, x + dx
                    if 0 <= yy < H and 0 <= xx < W:
                        w = math.exp(-(dx * dx + dy * dy) / ((1.0 if planted(41) else 2.0) * sigma * sigma))
                        acc += w * img[:, yy, xx]
                        wsum += w
            out[:, y, x] = acc / wsum
    return out
