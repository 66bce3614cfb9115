"""Pins of the oracle's progressive-resolution and blur schedules (Sec. 3.3
"Progressive Training", "Blur"; Sec. 4.1): schedule end points and midpoints,
the area resize against block means and a hand example, the blur against a
Gaussian's closed form and a separable restatement. CPU only."""
import math

import numpy as np
import pytest

from oracle import image_schedules as IS


def test_resolution_schedule():
    assert IS.scale_at(0) == pytest.approx(0.175)
    assert IS.scale_at(3000) == pytest.approx(0.175 + 0.825 / 2)
    assert IS.scale_at(6000) == 1.0 and IS.scale_at(9000) == 1.0
    s = [IS.scale_at(k) for k in range(0, 6001, 100)]
    assert all(b >= a for a, b in zip(s, s[1:]))
    assert IS.size_at(0, 1237, 822) == (216, 144)  # 0.175 * (1237, 822) = (216.475, 143.85)
    assert IS.size_at(6000, 1237, 822) == (1237, 822)


def test_blur_schedule():
    assert IS.sigma_at(0) == pytest.approx(1.0)
    assert IS.sigma_at(3000) == pytest.approx(0.5)
    assert IS.sigma_at(6000) == pytest.approx(0.0, abs=1e-15)


def test_area_resize_integer_factor_is_block_mean():
    g = np.random.default_rng(0)
    img = g.uniform(0, 1, (3, 8, 12))
    got = IS.resize_area(img, 6, 4)
    want = img.reshape(3, 4, 2, 6, 2).mean(axis=(2, 4))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


def test_area_resize_hand_example_and_constants():
    # 3 -> 2 pixels: r = 2/3; target 0 covers [-0.5, 1.0): source 0 over 1,
    # source 1 over 0.5 -> (2/3, 1/3); target 1 covers [1.0, 2.5): source 1
    # over 0.5, source 2 over 1 -> (1/3, 2/3)
    np.testing.assert_allclose(IS.area_weights(3, 2), [[2 / 3, 1 / 3, 0.0], [0.0, 1 / 3, 2 / 3]], atol=1e-15)
    # 1-D projection consistency: the source centre u maps to (u + 1/2) r - 1/2
    fx2, fy2, cx2, cy2 = IS.camera_at(1000.0, 900.0, 618.5, 411.0, 1237, 822, 216, 144)
    assert fx2 == pytest.approx(1000.0 * 216 / 1237) and cx2 == pytest.approx((618.5 + 0.5) * 216 / 1237 - 0.5)
    c = np.full((3, 37, 53), 0.3)
    np.testing.assert_allclose(IS.resize_area(c, 9, 7), 0.3, atol=1e-15)
    x = np.random.default_rng(1).uniform(0, 1, (3, 5, 7))
    np.testing.assert_allclose(IS.resize_area(x, 7, 5), x, atol=1e-15)  # scale 1: identity


def test_blur_delta_constant_identity_and_separable():
    H = W = 15
    d = np.zeros((1, H, W))
    d[0, 7, 7] = 1.0
    s = 0.8
    got = IS.blur(d, s)
    w = np.array([math.exp(-(k * k) / (2 * s * s)) for k in range(-2, 3)])
    k2 = np.outer(w, w) / np.outer(w, w).sum()
    np.testing.assert_allclose(got[0, 5:10, 5:10], k2, atol=1e-15)
    assert np.abs(got[0]).sum() == pytest.approx(1.0)
    c = np.full((3, 6, 9), 0.7)
    np.testing.assert_allclose(IS.blur(c, 1.0), 0.7, atol=1e-15)  # renormalised at the borders
    x = np.random.default_rng(2).uniform(0, 1, (3, 6, 9))
    assert np.array_equal(IS.blur(x, 0.05), x)
    # separable restatement with border renormalisation
    def blur1d(a, axis):
        n = a.shape[axis]
        out = np.zeros_like(a)
        for i in range(n):
            idx = [j for j in range(i - 2, i + 3) if 0 <= j < n]
            ww = np.array([math.exp(-((j - i) ** 2) / (2 * 1.3 * 1.3)) for j in idx])
            out.swapaxes(0, axis)[i] = np.tensordot(ww / ww.sum(), a.swapaxes(0, axis)[idx], axes=1)
        return out
    y = blur1d(blur1d(x, 1), 2)
    np.testing.assert_allclose(IS.blur(x, 1.3), y, atol=1e-14)
