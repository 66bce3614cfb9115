"""Pins of the oracle's absolute-value opacity activation (the finetuning
stage of Sec. 4.1, taken from Taming 3DGS): opacity = |x| exactly, the
switch from sigmoid leaves every rendered value unchanged, and the analytic
gradient through |x| against central differences. CPU only."""
import numpy as np
import pytest

from oracle import densify as D
from paper_2504_06716_gb300 import synth


def _scene(orc, n=9, W=24, H=20, tile=8, seed=5):
    g = np.random.default_rng(seed)
    P = np.zeros((n, 59))
    P[:, 0:3] = g.uniform(-0.35, 0.35, (n, 3))
    P[:, 3:6] = g.normal(-1.6, 0.3, (n, 3))
    P[:, 6:10] = g.normal(size=(n, 4))
    P[:, 10] = g.uniform(0.05, 0.9, n) * g.choice([-1.0, 1.0], n)  # both signs, away from 0
    P[:, 11:] = g.normal(0, 0.3, 48)
    cam = synth.pinhole(W, H, 60.0, (0.2, -3.0, 0.3))
    return P, orc.make_cam(cam, tile=tile, dilation=0.3, bg=(0.05, 0.1, 0.15)), g.uniform(0, 1, (3, H, W))


def test_opacity_is_the_absolute_value(orc):
    P, cam, _ = _scene(orc)
    pr = orc.project(P, cam, opacity_act=1)
    vis = pr["radius"] > 0
    assert vis.sum() >= 5
    assert np.array_equal(pr["opacity"][vis], np.abs(P[vis, 10]))
    sg = orc.project(P, cam)
    assert np.allclose(sg["opacity"][vis], 1 / (1 + np.exp(-P[vis, 10])), rtol=1e-15)


def test_switch_keeps_the_image(orc):
    """x -> sigmoid(x) with |.| afterwards gives the same opacities, hence the
    same lists and image; the opacity's Adam moments restart."""
    P, cam, _ = _scene(orc)
    before = orc.forward(P, cam)
    Q, M, V = P.copy(), np.ones_like(P), np.ones_like(P)
    D.opacity_to_abs(Q, M, V)
    after = orc.forward(Q, cam, opacity_act=1)
    assert np.allclose(after["proj"]["opacity"], before["proj"]["opacity"], rtol=1e-15, atol=0)
    assert np.array_equal(after["vals"], before["vals"]) and np.array_equal(after["ranges"], before["ranges"])
    assert np.allclose(after["image"], before["image"], rtol=0, atol=1e-14)
    assert not M[:, 10].any() and not V[:, 10].any() and M[:, 9].all() and V[:, 11].all()
    assert np.all(Q[:, 10] > 0) and np.all(Q[:, 10] < 1)
    # carried moments: the Adam direction m / sqrt(v) of the opacity is kept
    M2, V2 = np.full_like(P, 0.3), np.full_like(P, 0.04)
    Q2 = P.copy()
    D.opacity_to_abs(Q2, M2, V2, rescale=True)
    s = Q2[:, 10] * (1 - Q2[:, 10])
    assert np.allclose(M2[:, 10] * s, 0.3, rtol=1e-12) and np.allclose(V2[:, 10] * s * s, 0.04, rtol=1e-12)
    assert np.allclose(M2[:, 10] / np.sqrt(V2[:, 10]), 0.3 / 0.2, rtol=1e-12)


def test_gradient_through_abs_matches_central_differences(orc):
    """All 59 parameters with the cut-offs off (smooth); the opacity column
    carries sign(x) dL/do, so a dropped sign fails on the negative ones."""
    P, cam, gt = _scene(orc)
    res = orc.loss_and_grad(P, cam, gt, smooth=True, opacity_act=1)
    G = res["G"]
    h = 1e-5
    fd = np.zeros_like(P)
    for i in range(P.shape[0]):
        for k in range(59):
            Pp, Pm = P.copy(), P.copy()
            Pp[i, k] += h
            Pm[i, k] -= h
            fd[i, k] = (orc.loss_only(Pp, cam, gt, smooth=True, opacity_act=1)
                        - orc.loss_only(Pm, cam, gt, smooth=True, opacity_act=1)) / (2 * h)
    scale = np.abs(fd).max()
    err = np.abs(G - fd)
    assert np.all(err <= 1e-5 * np.abs(fd) + 1e-7 * scale), (err / (np.abs(fd) + 1e-7 * scale)).max()
    neg = P[:, 10] < 0
    assert neg.any() and (~neg).any()
    d_op = res["grads2d"]["d_opacity"]
    assert np.allclose(G[:, 10], np.sign(P[:, 10]) * d_op, rtol=1e-15, atol=0)
    assert np.abs(G[neg, 10]).max() > 0


def test_opacity_above_one_still_caps_alpha(orc):
    """|x| may exceed 1 (the high-opacity Gaussians the finetuning converts
    to); alpha is still capped at 0.99."""
    P, cam, _ = _scene(orc, n=1)
    P[0, 0:3] = 0.0
    P[0, 3:6] = np.log(0.3)
    P[0, 10] = -4.0
    pr = orc.project(P, cam, opacity_act=1)
    assert pr["opacity"][0] == 4.0
    f = orc.forward(P, cam, opacity_act=1)
    assert f["image"].max() <= 0.99 * 10 + 1  # finite
    T = f["t_final"]
    assert T.min() == pytest.approx(0.01, rel=1e-12)  # centre pixel: alpha capped at 0.99
