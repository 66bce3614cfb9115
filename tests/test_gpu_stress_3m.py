"""Differentiation at the stress size: 3,000,000 Gaussians of the surface
generator (SH degree 3, float32) at 1920x1080, through the autograd wrappers
(autograd.rasterize -> crop -> autograd.ssim_l1_loss -> backward).

The loss is Eq. 3 on the 256x256 crop at the image centre, so the whole
1920x1080 rasteriser backward runs at full size while the FP64 oracle only
has to evaluate the Gaussians whose tile rectangles meet the crop (the set S;
every other Gaussian must get an exactly zero gradient). Checked:

* the crop image and the loss against the oracle;
* the full 59-parameter gradient of every Gaussian against the oracle's
  analytic gradient (same tolerances and ambiguity bounds as the smaller
  end-to-end tests);
* central finite differences of the FP64 oracle loss, h = 1e-3, on 64
  random parameters of each type (mean, log-scale, rotation, opacity, SH)
  among the Gaussians that contribute to the crop. The loss is piecewise
  smooth (tile lists, alpha floor and cap, transmittance stop), and a step
  of 1e-3 in a mean moves a Gaussian ~0.4 px here, across such decisions;
  the differences are therefore taken with every decision held at the
  point's values (tests/fd_util.py, oracle.render_pixels_locked), which
  converges to the derivative the backward computes. For SH coefficients,
  which no decision depends on, the plain differences are checked as well.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2504_06716_gb300 import autograd, lib, synth  # noqa: E402

import fd_util  # noqa: E402
import parity_util as pu  # noqa: E402

pytestmark = pytest.mark.gpu

N, W, H, TILE = 3_000_000, 1920, 1080, 16
X0, Y0, CS = 832, 416, 256  # the centred 256x256 crop, aligned to 32
TYPES = {"mean": (0, 3), "log_scale": (3, 6), "rotation": (6, 10), "opacity": (10, 11), "sh": (11, 59)}


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06716_gb300 import build

    build.build()
    oracle.build()
    lib.load()
    cam = pu.round_camera(synth.hemisphere_cameras(150, 4.0, W, H, 60.0)[0])
    ocam, gcam = pu.cameras(cam, tile=TILE)
    P = pu.f32(synth.gaussians_surface(N, 30))
    proj = oracle.project(P, ocam)
    nudge = np.random.default_rng(32)
    for _ in range(20):  # keep every projection decision out of float32's reach
        bad = np.nonzero(proj["margin"] <= pu.PROJ_MARGIN)[0]
        if len(bad) == 0:
            break
        # a tile-rectangle edge sits at mean +- radius: move the mean a little, and the scale
        P[bad, 0:3] = pu.f32(P[bad, 0:3] + nudge.normal(0.0, 2e-4, (len(bad), 3)))
        P[bad, 3:6] = pu.f32(P[bad, 3:6] + 3e-3)
        sub = oracle.project(P[bad], ocam)
        for k in proj:
            proj[k][bad] = sub[k]
    else:
        raise AssertionError("nudge failed")
    R = proj["rect"]
    S = np.nonzero((proj["radius"] > 0) & (R[:, 0] < (X0 + CS) // TILE) & (R[:, 2] > X0 // TILE)
                   & (R[:, 1] < (Y0 + CS) // TILE) & (R[:, 3] > Y0 // TILE))[0]
    gt = synth.smooth_image(CS, CS, 31)

    # GPU: the full-size forward and backward through the autograd wrappers
    Pt = torch.from_numpy(pu.pack64(P)).cuda().requires_grad_(True)
    image = autograd.rasterize(Pt, gcam)
    crop = image[:, Y0:Y0 + CS, X0:X0 + CS]
    loss = autograd.ssim_l1_loss(crop.contiguous(), torch.from_numpy(gt.astype(np.float32)).cuda())
    loss.backward()
    assert lib.gs_get_device_error() == 0
    G = Pt.grad.cpu().numpy()
    gpu_crop = crop.detach().cpu().numpy().astype(np.float64)
    gpu_loss = float(loss.item())
    del Pt, image, crop, loss
    torch.cuda.empty_cache()

    # oracle on the set S
    projS = {k: v[S] for k, v in proj.items()}
    PS = P[S]
    vals, ranges = oracle.sort(projS["mean2d"].astype(np.float32), projS["radius"], projS["depth"].astype(np.float32),
                               W, H, TILE)
    yy, xx = np.meshgrid(np.arange(Y0, Y0 + CS), np.arange(X0, X0 + CS), indexing="ij")
    ren = oracle.render_pixels(projS, vals, ranges, ocam, xx.ravel(), yy.ravel())
    img = ren["image"].reshape(3, CS, CS)
    L, dimg = oracle.loss(img, gt)
    dl = np.zeros((3, H, W))
    dl[:, Y0:Y0 + CS, X0:X0 + CS] = dimg
    amb = np.zeros((H, W), np.uint8)
    amb[Y0:Y0 + CS, X0:X0 + CS] = (ren["margin"] <= pu.E2E_PIXEL_MARGIN).reshape(CS, CS)
    tx = (W + TILE - 1) // TILE
    tile_mask = np.zeros(tx * ((H + TILE - 1) // TILE), np.uint8)
    for ty in range(Y0 // TILE, (Y0 + CS) // TILE):
        tile_mask[ty * tx + X0 // TILE: ty * tx + (X0 + CS) // TILE] = 1
    rb = oracle.render_bwd(projS, vals, ranges, ocam, dl, amb=amb, tile_mask=tile_mask)
    GS = oracle.project_bwd(PS, ocam, rb)["G"]
    bound = pu.param_bound(PS, ocam, rb["amb_abs"])
    return dict(cam=cam, ocam=ocam, P=P, S=S, PS=PS, projS=projS, gt=gt, G=G, gpu_crop=gpu_crop, gpu_loss=gpu_loss,
                img=img, L=L, amb=amb[Y0:Y0 + CS, X0:X0 + CS].astype(bool), GS=GS, bound=bound)


def test_crop_image_and_loss_match_oracle(case):
    c = case
    assert len(c["S"]) > 20000
    ok = ~np.broadcast_to(c["amb"], c["img"].shape)
    assert pu.close(c["gpu_crop"], c["img"], 1e-4, 1.0, mask=ok)[0]
    assert c["amb"].mean() < 0.02  # ambiguous pixels are rare and only checked for validity
    assert np.isfinite(c["gpu_crop"]).all() and (c["gpu_crop"] >= 0).all()
    assert c["gpu_loss"] == pytest.approx(c["L"], rel=1e-4)


def test_full_gradient_matches_oracle_on_the_crop(case):
    c = case
    G, S = c["G"], c["S"]
    outside = np.ones(N, bool)
    outside[S] = False
    assert not G[outside].any()  # Gaussians that cannot reach the crop get nothing
    assert not G[:, 59:].any()
    GS, bound = c["GS"], c["bound"]
    for name, (lo, hi) in TYPES.items():
        w = GS[:, lo:hi]
        good, worst = pu.close_bound(G[S, lo:hi], w, 1e-3, 1e-2 * np.abs(w).max(), bound[:, lo:hi])
        assert good, (name, worst)


def test_central_differences_on_64_parameters_per_type(case):
    c = case
    GS, bound, Gg = c["GS"], c["bound"], c["G"][c["S"]]
    g = np.random.default_rng(33)
    picks = {}
    for name, (lo, hi) in TYPES.items():
        blk = np.abs(GS[:, lo:hi])
        # contributors whose gradient is not dominated by float32-ambiguous pixels
        cand = np.nonzero((blk.max(axis=1) > 0) & (bound[:, lo:hi].max(axis=1) <= 1e-3 * blk.max(axis=1)))[0]
        assert len(cand) >= 64, name
        rows = g.choice(cand, 64, replace=False)
        picks[name] = [(int(i), int(g.integers(lo, hi))) for i in rows]
    state = dict(P=c["PS"], proj=c["projS"], cam=c["cam"], tile=TILE, crop=(X0, Y0, CS), gt=c["gt"])
    tasks = [(i, j, [1e-3], True) for name in TYPES for i, j in picks[name]]
    tasks += [(i, j, [1e-3], False) for i, j in picks["sh"]]
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, min(16, os.cpu_count() or 1)), initializer=fd_util.init, initargs=(state,)) as pool:
        res = pool.map(fd_util.local_fd, tasks)
    fd_locked = {}
    k = 0
    for name in TYPES:
        fd_locked[name] = np.array([res[k + q][0] for q in range(64)])
        k += 64
    fd_plain_sh = np.array([res[k + q][0] for q in range(64)])
    report = {}
    for name, (lo, hi) in TYPES.items():
        idx = picks[name]
        fd = fd_locked[name]
        gpu = np.array([Gg[i, j] for i, j in idx])
        orc = np.array([GS[i, j] for i, j in idx])
        bnd = np.array([bound[i, j] for i, j in idx])
        scale = np.abs(GS[:, lo:hi]).max()
        # h = 1e-3 truncation: up to ~1% for means (0.4 px steps), far less for the others
        tol = 1e-2 * np.abs(fd) + 1e-4 * scale + bnd
        err_gpu = np.abs(gpu - fd)
        err_orc = np.abs(orc - fd)
        report[name] = (float(np.median(err_gpu / (np.abs(fd) + 1e-4 * scale))), float((err_gpu / tol).max()))
        assert (err_orc <= tol).all(), (name, float((err_orc / tol).max()))
        assert (err_gpu <= tol).all(), (name, float((err_gpu / tol).max()))
    sh = picks["sh"]
    gpu_sh = np.array([Gg[i, j] for i, j in sh])
    scale = np.abs(GS[:, 11:59]).max()
    assert (np.abs(gpu_sh - fd_plain_sh) <= 1e-3 * np.abs(fd_plain_sh) + 1e-5 * scale).all()
    print("median relative error of the GPU gradient against the differences, worst ratio to tolerance:", report)
