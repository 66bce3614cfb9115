"""The local finite differences used by the 3M-Gaussian test equal plain
central differences of the whole crop's loss (CPU, small scene)."""
import numpy as np
import pytest

import oracle
from paper_2504_06716_gb300 import synth

import fd_util
import parity_util as pu


def _crop_loss(P, ocam, crop, gt):
    x0, y0, cs = crop
    f = oracle.project(P, ocam)
    vals, ranges = oracle.sort_proj(f, ocam.width, ocam.height, ocam.tile)
    yy, xx = np.meshgrid(np.arange(y0, y0 + cs), np.arange(x0, x0 + cs), indexing="ij")
    ren = oracle.render_pixels(f, vals, ranges, ocam, xx.ravel(), yy.ravel())
    return oracle.loss(ren["image"].reshape(3, cs, cs), gt, grad=False)[0]


def test_local_fd_equals_whole_crop_fd(orc):
    cam = pu.round_camera(synth.hemisphere_cameras(5, 4.0, 320, 240, 60.0)[2])
    P = pu.f32(synth.gaussians_surface(4000, 12))
    crop = (96, 64, 128)
    gt = synth.smooth_image(128, 128, 3)
    ocam = oracle.make_cam(cam, tile=16)
    proj = oracle.project(P, ocam)
    x0, y0, cs = crop
    R = proj["rect"]
    S = np.nonzero((proj["radius"] > 0) & (R[:, 0] < (x0 + cs) // 16) & (R[:, 2] > x0 // 16)
                   & (R[:, 1] < (y0 + cs) // 16) & (R[:, 3] > y0 // 16))[0]
    PS = P[S]
    fd_util.init(dict(P=PS, proj={k: v[S] for k, v in proj.items()}, cam=cam, tile=16, crop=crop, gt=gt))
    g = np.random.default_rng(0)
    h = 1e-3
    checked = 0
    for _ in range(12):
        i = int(g.integers(len(S)))
        j = int(g.choice([0, 4, 7, 10, 11, 30]))
        local = fd_util.local_fd((i, j, [h]))[0]
        Pp, Pm = PS.copy(), PS.copy()
        Pp[i, j] += h
        Pm[i, j] -= h
        full = (_crop_loss(Pp, ocam, crop, gt) - _crop_loss(Pm, ocam, crop, gt)) / (2 * h)
        assert local == pytest.approx(full, rel=1e-7, abs=1e-12), (i, j)
        checked += abs(full) > 0
    assert checked >= 6


def _small_case():
    cam = pu.round_camera(synth.hemisphere_cameras(5, 4.0, 320, 240, 60.0)[2])
    P = pu.f32(synth.gaussians_surface(4000, 12))
    crop = (96, 64, 128)
    gt = synth.smooth_image(128, 128, 3)
    ocam = oracle.make_cam(cam, tile=16)
    proj = oracle.project(P, ocam)
    x0, y0, cs = crop
    R = proj["rect"]
    S = np.nonzero((proj["radius"] > 0) & (R[:, 0] < (x0 + cs) // 16) & (R[:, 2] > x0 // 16)
                   & (R[:, 1] < (y0 + cs) // 16) & (R[:, 3] > y0 // 16))[0]
    projS = {k: v[S] for k, v in proj.items()}
    return cam, ocam, P[S], projS, crop, gt


def test_locked_render_records_and_replays_the_plain_render(orc):
    cam, ocam, P, proj, crop, gt = _small_case()
    vals, ranges = oracle.sort_proj(proj, ocam.width, ocam.height, 16)
    x0, y0, cs = crop
    yy, xx = np.meshgrid(np.arange(y0, y0 + cs), np.arange(x0, x0 + cs), indexing="ij")
    plain = oracle.render_pixels(proj, vals, ranges, ocam, xx.ravel(), yy.ravel())["image"]
    rec, dec = oracle.render_pixels_locked(proj, vals, ranges, ocam, xx.ravel(), yy.ravel())
    assert np.array_equal(rec, plain)
    rep, _ = oracle.render_pixels_locked(proj, vals, ranges, ocam, xx.ravel(), yy.ravel(), dec)
    assert np.array_equal(rep, plain)
    assert (dec == 0).any() and (dec == 1).any()  # both skips and blends occur


def test_locked_fd_equals_the_analytic_gradient(orc):
    """With decisions held, central differences converge to the oracle's
    analytic gradient (cut-offs on) for every kind of parameter."""
    cam, ocam, P, proj, crop, gt = _small_case()
    x0, y0, cs = crop
    vals, ranges = oracle.sort_proj(proj, ocam.width, ocam.height, 16)
    yy, xx = np.meshgrid(np.arange(y0, y0 + cs), np.arange(x0, x0 + cs), indexing="ij")
    img = oracle.render_pixels(proj, vals, ranges, ocam, xx.ravel(), yy.ravel())["image"].reshape(3, cs, cs)
    _, dimg = oracle.loss(img, gt)
    dl = np.zeros((3, ocam.height, ocam.width))
    dl[:, y0:y0 + cs, x0:x0 + cs] = dimg
    G = oracle.project_bwd(P, ocam, oracle.render_bwd(proj, vals, ranges, ocam, dl))["G"]
    fd_util.init(dict(P=P, proj=proj, cam=cam, tile=16, crop=crop, gt=gt))
    g = np.random.default_rng(1)
    for lo, hi in [(0, 3), (3, 6), (6, 10), (10, 11), (11, 59)]:
        cand = np.nonzero(np.abs(G[:, lo:hi]).max(axis=1) > 0)[0]
        scale = np.abs(G[:, lo:hi]).max()
        for _ in range(6):
            i, j = int(g.choice(cand)), int(g.integers(lo, hi))
            fd = fd_util.local_fd((i, j, [1e-5], True))[0]
            assert fd == pytest.approx(G[i, j], rel=1e-4, abs=1e-6 * scale), (i, j)
