"""Pins of the oracle's volume masks (Sec. 3.3, "Pruning with Volume
Masking"): the hard mask culls at logit(0.01) in float32, a mask that is on
changes nothing, the straight-through gradient of the mask logit equals the
central difference of the loss under a common scaling of opacity and scales
(what the mask multiplies), and pruning removes masked-off Gaussians. CPU only."""
import math

import numpy as np
import pytest

from oracle import densify as D
from paper_2504_06716_gb300 import synth

LOGIT_MIN = float(np.float32(math.log(0.01 / 0.99)))


def _scene(orc, n=9, W=24, H=20, tile=8, seed=5):
    g = np.random.default_rng(seed)
    P = np.zeros((n, 59))
    P[:, 0:3] = g.uniform(-0.35, 0.35, (n, 3))
    P[:, 3:6] = g.normal(-1.6, 0.3, (n, 3))
    P[:, 6:10] = g.normal(size=(n, 4))
    P[:, 10] = g.uniform(-1.0, 1.5, n)
    P[:, 11:] = g.normal(0, 0.3, 48)
    cam = synth.pinhole(W, H, 60.0, (0.2, -3.0, 0.3))
    return P, orc.make_cam(cam, tile=tile, dilation=0.3, bg=(0.05, 0.1, 0.15)), g.uniform(0, 1, (3, H, W))


def test_hard_mask_culls_at_the_float32_threshold(orc):
    P, cam, _ = _scene(orc)
    base = orc.project(P, cam)
    vis = base["radius"] > 0
    assert vis.sum() >= 6
    edge = np.float32(LOGIT_MIN)
    mask = np.full(P.shape[0], 2.0)
    mask[0], mask[1] = float(edge), float(np.nextafter(edge, np.float32(1)))
    mask[2] = -10.0
    pr = orc.project(P, cam, mask=mask)
    assert pr["radius"][0] == 0 and pr["radius"][2] == 0 and pr["opacity"][0] == 0
    on = np.ones(P.shape[0], bool)
    on[[0, 2]] = False
    for k in ("radius", "mean2d", "conic", "opacity", "rgb"):
        assert np.array_equal(pr[k][on], base[k][on]), k


def test_straight_through_gradient_is_the_common_scaling_derivative(orc):
    """dL/dM at M = 1 is d/dt L(o t, s t) at t = 1; G_mask = (dL/dM + mask_loss) sigmoid'(m)."""
    P, cam, gt = _scene(orc, seed=7)
    n = P.shape[0]
    mask = np.random.default_rng(1).uniform(-2.0, 3.0, n)
    mask[3] = -9.0  # off: only the mask term reaches it
    frozen = np.zeros(n, np.uint8)
    frozen[5] = 1
    lam = 0.37
    f = orc.forward(P, cam, smooth=True)
    L, dimg = orc.loss(f["image"], gt)
    g2 = orc.render_bwd(f["proj"], f["vals"], f["ranges"], cam, dimg, smooth=True)
    res = orc.project_bwd(P, cam, g2, frozen=frozen, smooth=True, mask=mask, mask_loss=lam)
    sm = 1 / (1 + np.exp(-mask))
    slope = sm * (1 - sm)
    o = 1 / (1 + np.exp(-P[:, 10]))
    h = 1e-6
    checked = 0
    for i in range(n):
        if i in (3, 5):
            continue
        def loss_t(t):
            Q = P.copy()
            ot = o[i] * t
            Q[i, 10] = math.log(ot / (1 - ot))
            Q[i, 3:6] += math.log(t)
            return orc.loss_only(Q, cam, gt, smooth=True)
        dM = (loss_t(1 + h) - loss_t(1 - h)) / (2 * h)
        assert res["G_mask"][i] == pytest.approx((dM + lam) * slope[i], rel=1e-5, abs=1e-10)
        checked += 1
    assert checked >= 6
    assert res["G_mask"][3] == pytest.approx(lam * slope[3], rel=1e-12)  # masked off: the mask term only
    assert res["G_mask"][5] == 0.0  # frozen: nothing


def test_mask_prune_decisions():
    P = np.zeros((4, 60), np.float32)
    P[:, 3:6] = math.log(0.01)
    P[:, 6] = 1.0
    P[:, 10] = 2.0
    edge = np.float32(LOGIT_MIN)
    P[:, 59] = [3.0, edge, np.nextafter(edge, np.float32(1)), -20.0]
    prm = D.DensifyParams(eps_xyz=1e9, eps_rgb=1e9, use_rgb=False, log_clone_max=math.log(0.044),
                          logit_min_opacity=D.logit(0.005), prune_big=False, max_screen_radius=20,
                          log_max_world=math.log(0.44), log_split_div=math.log(1.6), mask_prune=True,
                          mask_logit_min=LOGIT_MIN)
    z = np.zeros((0, 2, 3))
    out = D.densify(P.astype(np.float64), np.zeros(4), np.zeros(4), np.zeros(4), np.zeros(4, int), prm, z)
    assert out["src"].tolist() == [0, 2]
    prm.mask_prune = False
    assert D.densify(P.astype(np.float64), np.zeros(4), np.zeros(4), np.zeros(4), np.zeros(4, int), prm,
                     z)["src"].tolist() == [0, 1, 2, 3]
