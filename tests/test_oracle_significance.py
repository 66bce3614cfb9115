"""Pins of the oracle's significance pruning (Sec. 3.3, after LightGaussian):
hit counts of a single Gaussian against its closed form, the score's volume
normaliser, the selection's count and tie order. CPU only."""
import math

import numpy as np

from oracle import significance as S
from paper_2504_06716_gb300 import synth


def test_hits_of_one_gaussian_are_the_pixels_above_the_alpha_floor(orc):
    """One isotropic Gaussian facing the camera: a pixel blends it iff
    o exp(-d^2 / (2 var)) >= 1/255 (no other cut-off applies)."""
    W = H = 40
    P = np.zeros((1, 59))
    P[0, 3:6] = math.log(0.2)
    P[0, 6] = 1.0
    P[0, 10] = 0.5
    cam = orc.make_cam(synth.pinhole(W, H, 60.0, (0.0, -3.0, 0.0)), tile=8, dilation=0.0)
    f = orc.forward(P, cam)
    pr = f["proj"]
    hits = S.hit_counts(pr, f["vals"], f["ranges"], cam, 1)
    a, b, c = pr["conic"][0]
    mx, my = pr["mean2d"][0]
    o = pr["opacity"][0]
    want = 0
    for py in range(H):
        for px in range(W):
            dx, dy = mx - px, my - py
            al = o * math.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy)
            want += al >= 1 / 255.0
    assert hits[0] == want and want > 20


def test_scores_and_selection():
    P = np.zeros((10, 59))
    P[:, 3] = np.log(np.arange(1, 11, dtype=np.float64))  # volumes 1 .. 10
    P[:, 10] = 0.0  # opacity 1/2
    hits = np.full(10, 4)
    s = S.scores(P, hits, beta=1.0, quantile=0.9)  # V_q = volume of rank 8 = 9
    np.testing.assert_allclose(s, 4 * 0.5 * np.arange(1, 11) / 9.0, rtol=1e-12)
    s0 = S.scores(P, hits, beta=0.0)
    assert np.all(s0 == 2.0)
    assert S.mark(s0, 0.35).tolist() == [1, 1, 1, 0, 0, 0, 0, 0, 0, 0]  # ties: lowest indices first
    assert S.mark(s, 0.0).sum() == 0 and S.mark(s, 1.0).sum() == 10
    m = S.mark(np.array([5.0, 1.0, 3.0, 2.0]), 0.5)
    assert m.tolist() == [0, 1, 0, 1]
