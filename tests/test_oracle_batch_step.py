"""Pins of the batched step's oracle (oracle/batch_step.py): several scenes,
several views of each per step (not in the paper; the reading is stated in
that module). CPU only.

* the scene's gradient is the gradient of the sum of its views' losses:
  central finite differences in smooth mode;
* every view in which a Gaussian is visible and unfrozen counts once in the
  freeze statistics;
* Adam's first two steps from zero moments follow their closed form at the
  scene's own step counter;
* scenes are independent: a scene's result does not depend on the others or
  on their order;
* one scene with one view is Algorithm 1's single step.
"""
import math

import numpy as np
import pytest

from paper_2504_06716_gb300 import synth


@pytest.fixture(scope="module")
def B(orc):
    from oracle import batch_step

    return batch_step


def _scene(orc, n, seed, W=40, H=32, views=(0, 2)):
    g = np.random.default_rng(seed)
    P = np.zeros((n, 59))
    P[:, 0:3] = g.uniform(-0.5, 0.5, (n, 3))
    P[:, 3:6] = g.normal(-2.2, 0.25, (n, 3))
    P[:, 6:10] = g.normal(size=(n, 4))
    P[:, 10] = g.uniform(-1.0, 1.5, n)
    P[:, 11:14] = g.uniform(0.0, 1.0, (n, 3))
    P[:, 14:] = g.normal(0, 0.05, (n, 45))
    P = P.astype(np.float32).astype(np.float64)
    cams = synth.circle_cameras(4, 3.0, W, H, 60.0)
    oc = [orc.make_cam(cams[v], tile=16) for v in views]
    gts = [synth.smooth_image(H, W, 70 + seed + v) for v in views]
    return dict(P=P, M=np.zeros_like(P), V=np.zeros_like(P), frozen=np.zeros(n, np.uint8),
                acc_x=np.zeros(n, np.float32), acc_r=np.zeros(n, np.float32), cnt=np.zeros(n, np.int32), step=0,
                lr=np.array([1.6e-3, 5e-3, 1e-3, 2.5e-2, 2.5e-3, 1.25e-4]), cams=oc, gts=gts, action=None,
                eps_xyz=0.0, eps_rgb=0.0)


def _copy(s):
    return {k: (v.copy() if isinstance(v, np.ndarray) else (list(v) if isinstance(v, list) else v))
            for k, v in s.items()}


def test_scene_gradient_is_the_gradient_of_the_summed_view_losses(orc, B):
    s = _scene(orc, 30, 1)
    n = s["P"].shape[0]
    P0 = s["P"].copy()
    res = B.scene_step(s["P"], s["M"], s["V"], s["frozen"], np.zeros(n), np.zeros(n), np.zeros(n, np.int64),
                       s["cams"], s["gts"], np.zeros(6), 1, smooth=True)
    G = res["G"]
    h = 1e-5
    g = np.random.default_rng(2)
    checked = 0
    for i in g.choice(n, 6, replace=False):
        for j in (0, 4, 7, 10, 11, 30):
            Pp, Pm = P0.copy(), P0.copy()
            Pp[i, j] += h
            Pm[i, j] -= h
            fd = sum(orc.loss_only(Pp, c, gt, smooth=True) - orc.loss_only(Pm, c, gt, smooth=True)
                     for c, gt in zip(s["cams"], s["gts"])) / (2 * h)
            assert G[i, j] == pytest.approx(fd, rel=2e-4, abs=1e-9), (i, j)
            checked += abs(fd) > 1e-7
    assert checked > 10


def test_statistics_count_each_view_once(orc, B):
    s = _scene(orc, 60, 3)
    s["frozen"][::5] = 1
    out = B.batch_step([s], 7)[0]
    n = s["P"].shape[0]
    want_c = np.zeros(n, np.int64)
    for v in out["views"]:
        want_c += (v["fwd"]["proj"]["radius"] > 0) & (s["frozen"] == 0)
    assert np.array_equal(s["cnt"], want_c)
    assert want_c.max() == 2 and (want_c == 2).sum() > 10
    assert np.all(s["acc_x"][s["frozen"] == 1] == 0) and np.all(s["cnt"][s["frozen"] == 1] == 0)
    both = want_c == 2
    want_x = out["views"][0]["xyz_norm"] + out["views"][1]["xyz_norm"]
    assert np.allclose(s["acc_x"][both], want_x[both], rtol=1e-15, atol=0)


def test_adam_closed_form_at_the_scene_counter(orc, B):
    """From zero moments, step 1 moves each parameter by lr sign(g); step 2 with
    gradients g1, g2 by lr (0.1 (0.9 g1 + g2) / 0.19) / sqrt((0.001 (0.999 g1^2 + g2^2)) / (1 - 0.999^2))."""
    s = _scene(orc, 40, 5)
    P0 = s["P"].copy()
    r1 = B.batch_step([s], 0)[0]
    g1 = r1["G"]
    nz = np.abs(g1) > 1e-5  # eps = 1e-15 negligible at 1e-9 relative
    lr = np.repeat(s["lr"], [3, 3, 4, 1, 3, 45])[None, :] * np.ones_like(P0)
    assert np.allclose((P0 - s["P"])[nz], (lr * np.sign(g1))[nz], rtol=1e-9, atol=0)
    P1 = s["P"].copy()
    r2 = B.batch_step([s], 1)[0]
    g2 = r2["G"]
    both = nz & (np.abs(g2) > 1e-5)
    m = 0.1 * (0.9 * g1 + g2) / (1 - 0.9 ** 2)
    v = 0.001 * (0.999 * g1 * g1 + g2 * g2) / (1 - 0.999 ** 2)
    assert s["step"] == 2
    assert np.allclose((P1 - s["P"])[both], (lr * m / (np.sqrt(v) + 1e-15))[both], rtol=1e-9, atol=0)


def test_scenes_are_independent(orc, B):
    a, b, c = _scene(orc, 25, 7), _scene(orc, 50, 8, views=(1, 3)), _scene(orc, 35, 9, views=(0,))
    a["frozen"][::3] = 1
    alone = _copy(b)
    B.batch_step([alone], 4)
    together = [_copy(a), _copy(b), _copy(c)]
    B.batch_step(together, 4)
    reordered = [_copy(c), _copy(b), _copy(a)]
    B.batch_step(reordered, 4)
    for key in ("P", "M", "V", "acc_x", "acc_r", "cnt"):
        assert np.array_equal(together[1][key], alone[key])
        assert np.array_equal(reordered[1][key], alone[key])
        assert np.array_equal(reordered[0][key], together[2][key])


def test_one_scene_one_view_is_the_single_step(orc, B):
    s = _scene(orc, 45, 11, views=(1,))
    s["frozen"][1::4] = 1
    P, M, V = s["P"].copy(), s["M"].copy(), s["V"].copy()
    res = orc.loss_and_grad(P, s["cams"][0], s["gts"][0], frozen=s["frozen"])
    orc.adam(P, res["G"], M, V, s["frozen"], s["lr"], 1)
    out = B.batch_step([s], 0)[0]
    assert np.array_equal(out["G"], res["G"]) and np.array_equal(s["P"], P) and np.array_equal(s["V"], V)
    assert out["losses"][0] == res["loss"]


def test_freeze_action_comes_before_the_views(orc, B):
    """An update freezes on the statistics gathered before the step, and the
    step's views are then differentiated on the new map: newly frozen rows get
    no gradient and keep their parameters."""
    s = _scene(orc, 60, 13)
    s["acc_x"][:] = np.float32(1e-3)
    s["acc_r"][:] = np.float32(1e-3)
    s["cnt"][:] = 1
    s["acc_x"][::2] = np.float32(1e-9)
    s["acc_r"][::2] = np.float32(1e-9)
    s["action"], s["eps_xyz"], s["eps_rgb"] = 0, 1e-6, 1e-6
    P0 = s["P"].copy()
    out = B.batch_step([s], 3)[0]
    assert np.all(s["frozen"][::2] == 1) and np.all(s["frozen"][1::2] == 0)
    assert np.array_equal(out["act"], np.arange(1, 60, 2, dtype=np.int32))
    assert np.all(out["G"][::2] == 0) and np.array_equal(s["P"][::2], P0[::2])
    assert math.isfinite(out["losses"][0])
