"""The seeded input generators draw what the workloads state: value
distributions of the Gaussian sets, the surface mix, camera rigs, view
splits and per-epoch view orders. CPU only; nothing here depends on the
method's arithmetic."""
import math

import numpy as np
import pytest

from paper_2504_06716_gb300 import synth


def _is_unit(q, tol=1e-12):
    return np.all(np.abs(np.linalg.norm(q, axis=1) - 1.0) < tol)


def test_uniform_set_distributions():
    """Tiny workload: means U[-1,1]^3, log-scales N(-3.5, 0.3), unit
    quaternions, opacity logits U(-2, 2), SH DC U(0, 1), higher bands N(0, 0.05)."""
    n = 40000
    p = synth.gaussians_uniform(n, 3)
    assert p.shape == (n, 59) and p.dtype == np.float64
    m = p[:, 0:3]
    assert m.min() >= -1.0 and m.max() <= 1.0
    assert np.allclose(m.mean(axis=0), 0.0, atol=0.02) and np.allclose(m.std(axis=0), 2 / math.sqrt(12), atol=0.01)
    s = p[:, 3:6]
    assert abs(s.mean() + 3.5) < 0.01 and abs(s.std() - 0.3) < 0.01
    assert _is_unit(p[:, 6:10])
    assert p[:, 10].min() >= -2.0 and p[:, 10].max() <= 2.0 and abs(p[:, 10].mean()) < 0.05
    sh = p[:, 11:].reshape(n, 16, 3)
    assert sh[:, 0].min() >= 0.0 and sh[:, 0].max() <= 1.0 and abs(sh[:, 0].mean() - 0.5) < 0.01
    assert abs(sh[:, 1:].std() - 0.05) < 0.002 and abs(sh[:, 1:].mean()) < 0.002


def _surface_distance(pts):
    """Distance of each point to the nearest of the three surface families:
    the unit sphere, the ground plane y = -1.2 and the band of box faces
    (boxes stand on the plane and are at most 0.6 high)."""
    d_sphere = np.abs(np.linalg.norm(pts, axis=1) - 1.0)
    d_plane = np.abs(pts[:, 1] + 1.2)
    in_box_band = (pts[:, 1] > -1.25) & (pts[:, 1] < -0.55) & (np.abs(pts[:, 0]) < 3.35) & (np.abs(pts[:, 2]) < 3.35)
    d_box = np.where(in_box_band, 0.0, np.inf)
    return d_sphere, d_plane, d_box


def test_surface_set_lies_on_the_surface_mix():
    """Mid/stress workloads: points on a unit sphere, the ground plane and 20
    boxes (area-weighted), N(0, 0.01) jitter, log-scales N(-4.5, 0.5)."""
    n = 40000
    p = synth.gaussians_surface(n, 5)
    d_sphere, d_plane, d_box = _surface_distance(p[:, 0:3])
    near = np.minimum(np.minimum(d_sphere, d_plane), d_box)
    assert np.all(near < 0.06)  # 6 sigma of the jitter
    # sphere share ~ its area over the total: 4 pi / (4 pi + 64 + box faces)
    on_sphere = np.mean(d_sphere < 0.05)
    assert 0.10 < on_sphere < 0.17
    # the plane spans [-4, 4]^2
    plane = d_plane < 0.05
    assert np.abs(p[plane, 0]).max() <= 4.06 and np.abs(p[plane, 2]).max() <= 4.06
    # jitter: points drawn on the sphere are N(0, 0.01) off it along every axis
    radial = np.linalg.norm(p[d_sphere < 0.05, 0:3], axis=1) - 1.0
    assert abs(radial.std() - 0.01) < 0.001
    s = p[:, 3:6]
    assert abs(s.mean() + 4.5) < 0.02 and abs(s.std() - 0.5) < 0.01
    assert _is_unit(p[:, 6:10])
    assert p[:, 10].min() >= -2.0 and p[:, 10].max() <= 2.0


def test_ground_truth_set_is_opaque_and_textured():
    p = synth.gaussians_surface(20000, 6, ground_truth=True)
    assert p[:, 10].min() >= 2.0 and p[:, 10].max() <= 4.0
    assert abs(p[:, 14:].std() - 0.03) < 0.002
    # the DC colour follows the position (low-frequency texture), not noise alone
    x = p[:, 0]
    c = np.corrcoef(p[:, 11], np.sin(1.7 * x + 0.3))[0, 1]
    assert c > 0.3


def test_seeded_and_reproducible():
    a = synth.gaussians_surface(3000, 7)
    b = synth.gaussians_surface(3000, 7)
    c = synth.gaussians_surface(3000, 8)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.array_equal(synth.gaussians_uniform(500, 1), synth.gaussians_uniform(500, 1))
    assert np.array_equal(synth.smooth_image(20, 30, 4), synth.smooth_image(20, 30, 4))


def _check_rig(cams, radius, W, H, fov):
    f = W / (2.0 * math.tan(math.radians(fov) / 2.0))
    for cam in cams:
        assert (cam.width, cam.height) == (W, H)
        assert cam.fx == pytest.approx(f) and cam.fy == pytest.approx(f)
        assert (cam.cx, cam.cy) == (W / 2.0, H / 2.0)
        R = np.asarray(cam.R)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12) and np.linalg.det(R) == pytest.approx(1.0)
        assert np.linalg.norm(cam.campos) == pytest.approx(radius)
        assert np.allclose(R @ cam.campos + cam.t, 0.0, atol=1e-12)  # the centre maps to the camera origin
        o = R @ np.zeros(3) + cam.t  # the world origin lies straight ahead, at depth radius
        assert np.allclose(o, [0.0, 0.0, radius], atol=1e-12)


def test_circle_rig():
    cams = synth.circle_cameras(8, 4.0, 128, 128, 60.0)
    _check_rig(cams, 4.0, 128, 128, 60.0)
    assert all(abs(c.campos[2]) < 1e-12 for c in cams)
    ang = sorted(math.atan2(c.campos[1], c.campos[0]) % (2 * math.pi) for c in cams)
    assert np.allclose(np.diff(ang), 2 * math.pi / 8)


def test_hemisphere_rig():
    cams = synth.hemisphere_cameras(200, 4.0, 1237, 822, 60.0)
    _check_rig(cams, 4.0, 1237, 822, 60.0)
    ys = np.array([c.campos[1] for c in cams])
    assert ys.min() > 0.0  # upper hemisphere only
    eyes = np.stack([c.campos for c in cams])
    d = np.linalg.norm(eyes[:, None] - eyes[None], axis=2) + np.eye(len(cams)) * 1e9
    assert d.min() > 0.2  # spread out, no two cameras on top of each other


def test_view_split_and_order():
    train, test, subset = synth.split_views(200, 0.1, 2)
    assert test == list(range(7, 200, 8))
    assert sorted(train + test) == list(range(200)) and not set(train) & set(test)
    assert len(subset) == round(0.1 * len(train)) and set(subset) <= set(train)
    assert synth.split_views(200, 0.1, 2) == (train, test, subset)
    order = synth.view_order(3 * len(train) + 5, train, 9)
    for e in range(3):  # every epoch is a permutation of the training views
        assert sorted(order[e * len(train):(e + 1) * len(train)]) == train
    assert order == synth.view_order(3 * len(train) + 5, train, 9)


def test_workload_shapes():
    sc = synth.tiny_scene(0)
    assert sc.init.shape == (2000, 59) and sc.gt.shape == (3000, 59)
    assert len(sc.cameras) == 8 and all((c.width, c.height) == (128, 128) for c in sc.cameras)
    mid = synth.surface_scene(1000, 1500, 200, 1237, 822)
    assert mid.init.shape == (1000, 59) and mid.gt.shape == (1500, 59) and len(mid.cameras) == 200
    assert len(mid.test_views) == 25 and len(mid.subset_views) == round(0.1 * 175)


def test_smooth_image_range():
    img = synth.smooth_image(64, 96, 1)
    assert img.shape == (3, 64, 96)
    for c in range(3):
        assert img[c].min() == pytest.approx(0.0, abs=1e-12) and img[c].max() == pytest.approx(1.0)
