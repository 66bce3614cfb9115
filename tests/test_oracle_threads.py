"""The oracle's parallel loops give the same bits on one host thread as on
all of them: every sum is taken in an order fixed by the data (per-row and
per-entry partial sums added in order), not by the threads. CPU only."""
import numpy as np

from paper_2504_06716_gb300 import synth


def test_one_thread_equals_all_threads(orc):
    g = np.random.default_rng(17)
    P = synth.gaussians_uniform(900, 5)
    P[:, 3:6] += 0.9
    P = P.astype(np.float32).astype(np.float64)
    cam = orc.make_cam(synth.pinhole(96, 70, 60.0, (0.2, -0.3, 3.0)), tile=16, bg=(0.1, 0.2, 0.3))
    gt = g.uniform(0, 1, (3, 70, 96))
    frozen = (g.uniform(size=900) < 0.3).astype(np.uint8)
    many = orc.max_threads()
    try:
        orc.set_threads(1)
        a = orc.loss_and_grad(P, cam, gt, frozen=frozen)
        orc.set_threads(max(many, 4))
        b = orc.loss_and_grad(P, cam, gt, frozen=frozen)
    finally:
        orc.set_threads(many)
    assert a["loss"] == b["loss"]
    for key in ("G", "xyz_norm", "rgb_norm", "dl_dimage"):
        assert np.array_equal(a[key], b[key]), key
    assert np.array_equal(a["fwd"]["image"], b["fwd"]["image"])
    assert np.array_equal(a["fwd"]["vals"], b["fwd"]["vals"])
    assert np.abs(a["G"]).max() > 0
