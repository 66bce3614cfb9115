"""Stage-by-stage parity of the CUDA path (through the C ABI) with the FP64
oracle, at sizes the oracle finishes in seconds that span many tiles and
ragged tails. Integer outputs (sort order, tile ranges, freeze map, active
list) must match bit for bit; floating outputs within the stated tolerances
(1e-4 relative on images, 1e-3 relative on gradients)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2504_06716_gb300 import lib, synth  # noqa: E402

import parity_util as pu  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06716_gb300 import build

    build.build()
    oracle.build()
    lib.load()


def _scene(kind: str):
    """(params (n,59) float32-valued, cameras) for a parity workload."""
    if kind == "tiny":  # the 2,000-Gaussian, 128x128 workload
        s = synth.tiny_scene()
        return pu.f32(s.init), s.cameras
    if kind == "ragged":  # ragged image (100x75) and Gaussian count
        P = synth.gaussians_uniform(1733, 17)
        P[:, 3:6] += 0.8
        cams = synth.circle_cameras(3, 3.5, 100, 75, 55.0)
        return pu.f32(P), cams
    if kind == "surface":  # surface mix at a mid resolution
        s = synth.surface_scene(6000, 10, 8, 320, 214, seed=5)
        return pu.f32(s.init), s.cameras
    raise KeyError(kind)


def _gpu_project(P, gcam, deg=3):
    n = P.shape[0]
    Pt = torch.from_numpy(pu.pack64(P)).to(DEV)
    spl = torch.zeros((n, 12), dtype=torch.float32, device=DEV)
    lib.gs_project(Pt, n, deg, gcam, spl)
    torch.cuda.synchronize()
    return spl.cpu().numpy()


def _gpu_sort(rec, gcam, capacity=None):
    n = rec.shape[0]
    if capacity is None:
        capacity = int(rec[:, 11].view(np.int32).astype(np.int64).sum()) + 7
    spl = torch.from_numpy(rec).to(DEV)
    ws = torch.zeros(lib.gs_sort_workspace_bytes(n, capacity, gcam), dtype=torch.uint8, device=DEV)
    vals = torch.full((max(capacity, 1),), -1, dtype=torch.int32, device=DEV)
    ranges = torch.full((gcam.tiles, 2), -1, dtype=torch.int32, device=DEV)
    count = torch.zeros(1, dtype=torch.int64, device=DEV)
    lib.gs_sort(spl, n, gcam, ws, capacity, vals, ranges, count)
    flags = lib.gs_get_device_error()
    P = int(count.item())
    return vals.cpu().numpy().view(np.uint32), ranges.cpu().numpy().view(np.uint32), P, flags, spl


def _gpu_render(spl_t, vals_np, ranges_np, gcam):
    H, W = gcam.height, gcam.width
    vals = torch.from_numpy(vals_np.view(np.int32).copy()).to(DEV)
    ranges = torch.from_numpy(ranges_np.view(np.int32).copy()).to(DEV)
    img = torch.zeros((3, H, W), device=DEV)
    tf = torch.zeros((H, W), device=DEV)
    nl = torch.zeros((H, W), dtype=torch.int32, device=DEV)
    lib.gs_render_fwd(spl_t, vals, ranges, gcam, img, tf, nl)
    torch.cuda.synchronize()
    return img.cpu().numpy(), tf.cpu().numpy(), nl.cpu().numpy(), vals, ranges


# ----------------------------------------------------------------------------- A1 projection


@pytest.mark.parametrize("kind", ["tiny", "ragged", "surface"])
def test_project_matches_oracle(kind):
    P, cams = _scene(kind)
    for cam in cams[:4]:
        ocam, gcam = pu.cameras(cam)
        want = oracle.project(P, ocam)
        got = _gpu_project(P, gcam)
        safe = want["margin"] > pu.PROJ_MARGIN
        rad = got[:, 10].view(np.int32)
        tt = got[:, 11].view(np.int32)
        assert safe.mean() > 0.95
        assert np.array_equal(rad[safe], want["radius"][safe])
        assert np.array_equal(tt[safe], want["tiles_touched"][safe])
        vis = safe & (want["radius"] > 0)
        assert vis.sum() > 50
        assert np.abs(got[vis, 0:2] - want["mean2d"][vis]).max() < 1e-3
        scale = np.maximum(np.abs(want["conic"][vis, 0]), np.abs(want["conic"][vis, 2]))[:, None]
        assert (np.abs(got[vis, 2:5] - want["conic"][vis]) / scale).max() < 1e-4
        assert np.allclose(got[vis, 5], want["opacity"][vis], rtol=1e-6, atol=0)
        assert np.abs(got[vis, 6:9] - want["rgb"][vis]).max() < 1e-5
        assert np.allclose(got[vis, 9], want["depth"][vis], rtol=1e-6, atol=0)
        # culled Gaussians are all-zero records
        culled = safe & (want["radius"] == 0)
        assert np.all(got[culled] == 0)


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_project_lower_sh_degrees(deg):
    P, cams = _scene("tiny")
    ocam, gcam = pu.cameras(cams[1])
    want = oracle.project(P, ocam, sh_degree=deg)
    got = _gpu_project(P, gcam, deg)
    vis = (want["margin"] > pu.PROJ_MARGIN) & (want["radius"] > 0)
    assert np.abs(got[vis, 6:9] - want["rgb"][vis]).max() < 1e-5


def test_project_empty_and_all_culled():
    _, gcam = pu.cameras(synth.tiny_scene().cameras[0])
    spl = torch.zeros((1, 12), device=DEV)
    lib.gs_project(torch.zeros((1, 64), device=DEV), 0, 3, gcam, spl)  # n = 0
    P = np.zeros((5, 59))
    P[:, 0:3] = [100.0, 100.0, 100.0]  # behind / far outside every camera
    P[:, 6] = 1.0
    got = _gpu_project(pu.f32(P), gcam)
    assert np.all(got == 0)


# ----------------------------------------------------------------------------- A2 sort (bit-exact)


def _oracle_sort(rec, ocam, capacity=None):
    return oracle.sort_records(rec, ocam.width, ocam.height, ocam.tile, capacity=capacity)


def _check(vals, ranges, Pn, want_vals, want_ranges, rec, gcam):
    """Lists against the oracle's (pu.check_lists); returns the CUDA-only entries."""
    assert Pn >= len(want_vals)
    extra = pu.check_lists(vals[:Pn], ranges, want_vals, want_ranges, rec, gcam.tile, gcam.tiles_x)
    assert extra <= 0.05 * max(len(want_vals), 1) + 8, (extra, len(want_vals))
    return extra


@pytest.mark.parametrize("kind,tile", [("tiny", 16), ("ragged", 8), ("ragged", 32), ("surface", 16), ("surface", 8)])
def test_sort_matches_oracle(kind, tile):
    P, cams = _scene(kind)
    ocam, gcam = pu.cameras(cams[0], tile=tile)
    rec = pu.records_from_oracle(oracle.project(P, ocam))
    want_vals, want_ranges = _oracle_sort(rec, ocam)
    vals, ranges, Pn, flags, _ = _gpu_sort(rec, gcam)
    assert flags == 0
    assert len(want_vals) > 0
    _check(vals, ranges, Pn, want_vals, want_ranges, rec, gcam)


def test_sort_ties_keep_index_order():
    """Many Gaussians with bit-identical depth on overlapping tiles: the order
    inside a tile must be ascending index (the stable-sort tie break)."""
    g = np.random.default_rng(0)
    n = 5000
    rec = np.zeros((n, 12), np.float32)
    rec[:, 0] = g.uniform(0, 200, n)
    rec[:, 1] = g.uniform(0, 120, n)
    rec[:, 9] = g.choice(np.array([1.5, 2.25, 3.0, 7.0], np.float32), n)
    rad = g.integers(1, 30, n).astype(np.int32)
    rad[::7] = 0  # some culled
    rec[:, 10] = rad.view(np.float32)
    # isotropic splats whose 3-sigma circle has the radius, opaque enough to be listed
    sig = np.maximum(rad, 1).astype(np.float32) / 3.0
    rec[:, 2] = rec[:, 4] = 1.0 / (sig * sig)
    rec[:, 5] = 0.9
    cam = synth.pinhole(200, 120, 60.0, (0, -3, 0.5))
    ocam, gcam = pu.cameras(cam, tile=16)
    listed = np.zeros(n, np.int32)
    for i in range(n):  # tiles listing the splat by the oracle's rule
        if rad[i] > 0:
            v, _ = oracle.sort_records(rec[i:i + 1], 200, 120, 16)
            listed[i] = len(v)
    rad[listed == 0] = 0
    rec[:, 10] = rad.view(np.float32)
    x0 = np.clip(np.floor((rec[:, 0] - rad) / 16), 0, None)
    x1 = np.clip(np.floor((rec[:, 0] + rad) / 16), None, (200 + 15) // 16 - 1)
    y0 = np.clip(np.floor((rec[:, 1] - rad) / 16), 0, None)
    y1 = np.clip(np.floor((rec[:, 1] + rad) / 16), None, (120 + 15) // 16 - 1)
    rect = np.where((rad > 0) & (x0 <= x1) & (y0 <= y1), (x1 - x0 + 1) * (y1 - y0 + 1), 0).astype(np.int32)
    rec[:, 11] = rect.view(np.float32)  # the projection's count: tiles of the rectangle
    want_vals, want_ranges = _oracle_sort(rec, ocam)
    vals, ranges, Pn, flags, _ = _gpu_sort(rec, gcam)
    assert flags == 0
    _check(vals, ranges, Pn, want_vals, want_ranges, rec, gcam)


@pytest.mark.parametrize("tile", [8, 16])
def test_sort_extreme_conics(tile):
    """Splats from needle-thin to round, at every orientation and opacities
    down to the listing floor: the lists (built from candidate tiles the
    conic's ellipse bounds) equal the oracle's, which tests every tile of the
    3-sigma rectangle."""
    g = np.random.default_rng(11)
    n = 6000
    W, H = 400, 260
    rec = np.zeros((n, 12), np.float32)
    rec[:, 0] = g.uniform(-30, W + 30, n)
    rec[:, 1] = g.uniform(-30, H + 30, n)
    rec[:, 9] = g.uniform(1.0, 9.0, n).astype(np.float32)
    # 2-D covariance with eigenvalues l1 >= l2 >= 0.3 (the dilation), condition up to 1e5
    l2 = g.uniform(0.3, 4.0, n)
    l1 = l2 * np.exp(g.uniform(0, np.log(1e5), n))
    l1 = np.minimum(l1, 80.0 ** 2)
    th = g.uniform(0, np.pi, n)
    cth, sth = np.cos(th), np.sin(th)
    sxx = l1 * cth * cth + l2 * sth * sth
    syy = l1 * sth * sth + l2 * cth * cth
    sxy = (l1 - l2) * cth * sth
    det = sxx * syy - sxy * sxy
    rec[:, 2] = syy / det
    rec[:, 3] = -sxy / det
    rec[:, 4] = sxx / det
    rec[:, 5] = np.exp(g.uniform(np.log(1 / 255.0), 0.0, n)).astype(np.float32)
    rad = np.ceil(3 * np.sqrt(l1)).astype(np.int32)
    cam = synth.pinhole(W, H, 60.0, (0, -3, 0.5))
    ocam, gcam = pu.cameras(cam, tile=tile)
    rec[:, 10] = rad.view(np.float32)
    tx, ty = (W + tile - 1) // tile, (H + tile - 1) // tile
    x0 = np.clip(np.floor((rec[:, 0] - rad) / tile), 0, None)
    x1 = np.clip(np.floor((rec[:, 0] + rad) / tile), None, tx - 1)
    y0 = np.clip(np.floor((rec[:, 1] - rad) / tile), 0, None)
    y1 = np.clip(np.floor((rec[:, 1] + rad) / tile), None, ty - 1)
    tt = np.where((x0 <= x1) & (y0 <= y1), (x1 - x0 + 1) * (y1 - y0 + 1), 0).astype(np.int32)
    rad[tt == 0] = 0
    rec[:, 10] = rad.view(np.float32)
    rec[:, 11] = tt.view(np.float32)
    want_vals, want_ranges = _oracle_sort(rec, ocam)
    vals, ranges, Pn, flags, _ = _gpu_sort(rec, gcam)
    assert flags == 0 and len(want_vals) > 1000
    _check(vals, ranges, Pn, want_vals, want_ranges, rec, gcam)


def test_sort_empty_input():
    P = np.zeros((300, 59))
    P[:, 2] = -50.0  # behind the camera
    P[:, 6] = 1.0
    ocam, gcam = pu.cameras(synth.pinhole(64, 64, 60.0, (0, -3, 0.5)))
    rec = pu.records_from_oracle(oracle.project(pu.f32(P), ocam))
    vals, ranges, Pn, flags, _ = _gpu_sort(rec, gcam, capacity=16)
    assert Pn == 0 and flags == 0
    assert np.all(ranges == 0)


def test_sort_capacity_overflow_is_flagged_and_clipped():
    P, cams = _scene("tiny")
    ocam, gcam = pu.cameras(cams[0])
    rec = pu.records_from_oracle(oracle.project(P, ocam))
    want_vals, _ = _oracle_sort(rec, ocam)
    cap = len(want_vals) // 2
    vals, ranges, Pn, flags, _ = _gpu_sort(rec, gcam, capacity=cap)
    assert flags & lib.GS_FLAG_CAPACITY
    assert Pn >= len(want_vals)
    assert ranges.max() <= cap
    # the device flag is sticky until read, and reading clears it
    assert lib.gs_get_device_error() == 0


def _random_records(n, W, H, tile, seed):
    """Isotropic splats scattered over a W x H image, radii 1-40 px, random
    depths; the tile count field is the 3-sigma rectangle's (the projection's)."""
    g = np.random.default_rng(seed)
    rec = np.zeros((n, 12), np.float32)
    rec[:, 0] = g.uniform(-20, W + 20, n)
    rec[:, 1] = g.uniform(-20, H + 20, n)
    rec[:, 9] = g.uniform(0.5, 30.0, n)
    rad = g.integers(1, 40, n).astype(np.int32)
    rec[:, 10] = rad.view(np.float32)
    sig = rad.astype(np.float32) / 3.0
    rec[:, 2] = rec[:, 4] = 1.0 / (sig * sig)
    rec[:, 5] = g.uniform(0.02, 0.99, n)
    tx, ty = (W + tile - 1) // tile, (H + tile - 1) // tile
    x0 = np.clip(np.floor((rec[:, 0] - rad) / tile), 0, None)
    x1 = np.clip(np.floor((rec[:, 0] + rad) / tile), None, tx - 1)
    y0 = np.clip(np.floor((rec[:, 1] - rad) / tile), 0, None)
    y1 = np.clip(np.floor((rec[:, 1] + rad) / tile), None, ty - 1)
    rect = np.where((x0 <= x1) & (y0 <= y1), (x1 - x0 + 1) * (y1 - y0 + 1), 0).astype(np.int32)
    rec[:, 11] = rect.view(np.float32)
    return rec


@pytest.mark.parametrize("W,H,tile", [(1600, 1400, 8), (1024, 1024, 8), (120, 90, 8)])
def test_sort_super_tile_grids(W, H, tile):
    """Grids of 550 super-tiles (two radix passes by super-tile id), 256 (one
    pass, its digit ranges taken as the segments) and 4."""
    rec = _random_records(12000 if W > 500 else 1500, W, H, tile, seed=W)
    ocam, gcam = pu.cameras(synth.pinhole(W, H, 60.0, (0, -3, 0.5)), tile=tile)
    want_vals, want_ranges = _oracle_sort(rec, ocam)
    vals, ranges, Pn, flags, _ = _gpu_sort(rec, gcam)
    assert flags == 0
    assert len(want_vals) > 0
    _check(vals, ranges, Pn, want_vals, want_ranges, rec, gcam)


@pytest.mark.parametrize("cap", [0, 5])
def test_sort_capacity_below_the_super_tile_entries(cap):
    """A capacity smaller than the super-tile entries themselves: the entry
    count is then taken tile by tile and must equal the full sort's."""
    rec = _random_records(3000, 320, 200, 8, seed=3)
    _, gcam = pu.cameras(synth.pinhole(320, 200, 60.0, (0, -3, 0.5)), tile=8)
    _, _, P_full, flags_full, _ = _gpu_sort(rec, gcam)
    assert flags_full == 0 and P_full > 100
    vals, ranges, Pn, flags, _ = _gpu_sort(rec, gcam, capacity=cap)
    assert flags & lib.GS_FLAG_CAPACITY
    assert Pn == P_full
    assert ranges.max() <= cap
    assert lib.gs_get_device_error() == 0


# ----------------------------------------------------------------------------- A3 render forward


@pytest.mark.parametrize("kind,tile,bg", [("tiny", 16, (0, 0, 0)), ("ragged", 8, (0.2, 0.4, 0.6)),
                                          ("ragged", 32, (0, 0, 0)), ("surface", 16, (0.1, 0.1, 0.1))])
def test_render_forward_matches_oracle(kind, tile, bg):
    P, cams = _scene(kind)
    ocam, gcam = pu.cameras(cams[0], tile=tile, bg=bg)
    rec = pu.records_from_oracle(oracle.project(P, ocam))
    proj = pu.proj_from_records(rec)
    vals, ranges, Pn, flags, spl = _gpu_sort(rec, gcam)
    want = oracle.render(proj, vals[:Pn], ranges, ocam)
    img, tf, nl, _, _ = _gpu_render(spl, vals[:Pn], ranges, gcam)
    ok = want["margin"] > pu.PIXEL_MARGIN
    assert ok.mean() > 0.99
    assert np.array_equal(nl[ok], want["n_last"][ok])
    good, worst = pu.close(img, want["image"], 1e-4, 1.0, np.broadcast_to(ok, img.shape))
    assert good, worst
    good, worst = pu.close(tf, want["t_final"], 1e-4, 1e-3, ok)
    assert good, worst
    # pixels with an ambiguous decision must still hold a valid composite
    assert np.all(np.isfinite(img)) and np.all((tf >= 1e-4 * 0.99) & (tf <= 1.0))


@pytest.mark.parametrize("kind,tile", [("tiny", 16), ("surface", 8)])
def test_pair_counts_match_oracle_decisions(kind, tile):
    """gs_raster_pair_counts (measurement support) against the oracle's own
    record of every decision, over the pairs the resuming backward walks:
    each pixel's list up to its last contributor or 1 + the tile's last
    unfrozen entry among the first (deepest contributor) ones, whichever is
    less; with no freeze map, up to the last contributor."""
    P, cams = _scene(kind)
    ocam, gcam = pu.cameras(cams[0], tile=tile)
    rec = pu.records_from_oracle(oracle.project(P, ocam))
    proj = pu.proj_from_records(rec)
    vals, ranges, Pn, flags, spl = _gpu_sort(rec, gcam)
    want = oracle.render(proj, vals[:Pn], ranges, ocam)
    _, _, nl, vt, rt = _gpu_render(spl, vals[:Pn], ranges, gcam)
    frozen = (np.random.default_rng(7).uniform(size=P.shape[0]) < 0.3).astype(np.uint8)
    counts = torch.zeros(3, dtype=torch.int64, device=DEV)
    lib.gs_raster_pair_counts(spl, vt, rt, gcam, torch.from_numpy(nl).to(DEV), torch.from_numpy(frozen).to(DEV),
                              counts)
    got = counts.cpu().numpy()
    H, W = ocam.height, ocam.width
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    _, dec = oracle.render_pixels_locked(proj, vals[:Pn], ranges, ocam, xx.ravel(), yy.ravel())
    tiles = (yy // tile) * ((W + tile - 1) // tile) + xx // tile
    starts = ranges[tiles.ravel(), 0].astype(np.int64)
    nlo = want["n_last"].ravel()
    pos = np.arange(dec.shape[1])[None, :]
    inside = pos < nlo[:, None]
    g = vals[np.minimum(starts[:, None] + pos, max(Pn - 1, 0))]
    blended = inside & ((dec == 1) | (dec == 2))
    # walked: up to min(n_last, 1 + the tile's last unfrozen entry below its deepest n_last)
    tl = tiles.ravel()
    maxnl = np.zeros(int(tl.max()) + 1, np.int64)
    np.maximum.at(maxnl, tl, nlo)
    lu = np.full(maxnl.shape[0], -1, np.int64)
    for t in np.nonzero(maxnl)[0]:
        e = frozen[vals[ranges[t, 0]:ranges[t, 0] + maxnl[t]]] == 0
        if e.any():
            lu[t] = int(np.nonzero(e)[0][-1])
    upto = np.minimum(nlo, lu[tl] + 1)
    need = pos < upto[:, None]
    want_c = np.array([(need & blended & (frozen[g] == 0)).sum(), (need & blended & (frozen[g] == 1)).sum(),
                       (need & inside & (dec == 0)).sum()])
    # pixels whose decisions are within float32 reach may count either way
    amb = (want["margin"] <= pu.PIXEL_MARGIN).ravel()
    slack = int(nlo[amb].sum() + nl.ravel()[amb].sum())
    assert np.abs(got - want_c).sum() <= slack, (got, want_c, slack)
    assert want_c.sum() < inside.sum()  # the freeze map leaves pairs out
    # with no freeze map: every pair up to each pixel's last contributor
    counts.zero_()
    lib.gs_raster_pair_counts(spl, vt, rt, gcam, torch.from_numpy(nl).to(DEV), None, counts)
    assert int(counts.sum().item()) == nl.astype(np.int64).sum()


# ----------------------------------------------------------------------------- A4 loss


def _gpu_loss(x, y, lam=0.2):
    H, W = x.shape[1], x.shape[2]
    xt = torch.from_numpy(x.astype(np.float32)).to(DEV)
    yt = torch.from_numpy(y.astype(np.float32)).to(DEV)
    ws = torch.zeros(lib.gs_loss_workspace_bytes(H, W), dtype=torch.uint8, device=DEV)
    loss = torch.zeros(1, device=DEV)
    dl = torch.zeros_like(xt)
    lib.gs_loss(xt, yt, H, W, lam, ws, loss, dl)
    torch.cuda.synchronize()
    return float(loss.item()), dl.cpu().numpy()


def test_loss_gradient_finite_where_the_ssim_covariance_term_vanishes():
    """n2 = 2 cov(x, y) + C2 crosses zero across the image (anti-correlated
    textures of growing strength): the SSIM map's partials stay finite there
    (m / n2 = n1 / (d1 d2)) and equal the oracle's."""
    H, W = 64, 256
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    u = np.sin(0.9 * xx + 1.3 * yy) * np.cos(0.7 * yy)  # a zero-mean texture
    amp = np.sqrt(np.linspace(0.0, 4.0 * 4.5e-4, W))[None, :]  # cov ~ -amp^2 var(u), var(u) ~ 1/4
    x = pu.f32(np.clip(0.5 + amp * u, 0, 1))
    y = pu.f32(np.clip(0.5 - amp * u, 0, 1))
    x, y = np.stack([x, x, x]), np.stack([y, y * 0.99, y])
    Lw, dw = oracle.loss(x, y)
    Lg, dg = _gpu_loss(x, y)
    assert np.isfinite(dg).all() and np.isfinite(Lg)
    assert Lg == pytest.approx(Lw, rel=1e-5)
    assert np.abs(dg - dw).max() <= 1e-4 * np.abs(dw).max()
    assert lib.gs_get_device_error() == 0


@pytest.mark.parametrize("H,W", [(37, 53), (128, 128), (75, 100)])
def test_loss_matches_oracle(H, W):
    g = np.random.default_rng(H * W)
    x = pu.f32(g.uniform(0, 1, (3, H, W)))
    y = pu.f32(np.clip(x + g.normal(0, 0.1, x.shape), 0, 1))
    Lw, dw = oracle.loss(x, y)
    Lg, dg = _gpu_loss(x, y)
    assert Lg == pytest.approx(Lw, rel=1e-5)
    scale = np.abs(dw).mean()
    good, worst = pu.close(dg, dw, 1e-3, scale)
    assert good, worst


def test_loss_on_rendered_images():
    """Smooth rendered content (small local variance) is the hard case for the
    float32 window moments."""
    P, cams = _scene("tiny")
    s = synth.tiny_scene()
    ocam, _ = pu.cameras(cams[2])
    x = pu.f32(oracle.forward(P, ocam)["image"])
    y = pu.f32(oracle.forward(pu.f32(s.gt), ocam)["image"])
    Lw, dw = oracle.loss(x, y)
    Lg, dg = _gpu_loss(x, y)
    assert Lg == pytest.approx(Lw, rel=1e-5)
    good, worst = pu.close(dg, dw, 1e-3, np.abs(dw).mean())
    assert good, worst


def test_loss_identical_images():
    x = pu.f32(np.random.default_rng(2).uniform(0, 1, (3, 40, 30)))
    Lg, dg = _gpu_loss(x, x)
    assert abs(Lg) < 1e-6
    assert np.abs(dg).max() < 1e-9


# ----------------------------------------------------------------------------- A5/A6 backward


def _stage_inputs(kind, tile=16, bg=(0, 0, 0), cam_index=0, frozen_frac=0.3, seed=0):
    P, cams = _scene(kind)
    ocam, gcam = pu.cameras(cams[cam_index], tile=tile, bg=bg)
    rec = pu.records_from_oracle(oracle.project(P, ocam))
    proj = pu.proj_from_records(rec)
    vals, ranges, Pn, _, spl = _gpu_sort(rec, gcam)
    fw = oracle.render(proj, vals[:Pn], ranges, ocam)
    g = np.random.default_rng(seed)
    gt = pu.f32(np.clip(fw["image"] + g.normal(0, 0.05, fw["image"].shape), 0, 1))
    _, dl = oracle.loss(fw["image"], gt)
    dl = pu.f32(dl)
    frozen = (g.uniform(0, 1, P.shape[0]) < frozen_frac).astype(np.uint8)
    return dict(P=P, ocam=ocam, gcam=gcam, rec=rec, proj=proj, vals=vals[:Pn], ranges=ranges, spl=spl, fw=fw, dl=dl,
                frozen=frozen, gt=gt)


def _gpu_raster_bwd(st):
    n = st["P"].shape[0]
    _, tf, nl, vals, ranges = _gpu_render(st["spl"], st["vals"], st["ranges"], st["gcam"])
    tft = torch.from_numpy(tf).to(DEV)
    nlt = torch.from_numpy(nl).to(DEV)
    dlt = torch.from_numpy(st["dl"].astype(np.float32)).to(DEV)
    fr = torch.from_numpy(st["frozen"]).to(DEV)
    g2 = torch.zeros((n, 12), device=DEV)
    lib.gs_raster_bwd(st["spl"], vals, ranges, st["gcam"], tft, nlt, dlt, fr, g2)
    torch.cuda.synchronize()
    return g2.cpu().numpy(), tf, nl


@pytest.mark.parametrize("kind,tile,bg", [("tiny", 16, (0, 0, 0)), ("ragged", 8, (0.3, 0.2, 0.1)),
                                          ("surface", 16, (0, 0, 0)), ("ragged", 32, (0, 0, 0))])
def test_raster_backward_matches_oracle(kind, tile, bg):
    st = _stage_inputs(kind, tile, bg)
    g2, _, _ = _gpu_raster_bwd(st)
    amb = (st["fw"]["margin"] <= pu.PIXEL_MARGIN).astype(np.uint8)
    want = oracle.render_bwd(st["proj"], st["vals"], st["ranges"], st["ocam"], st["dl"], st["frozen"], amb)
    fr = st["frozen"] == 1
    assert np.all(g2[fr] == 0), "frozen Gaussians must receive nothing"
    a = ~fr
    W9 = pu.grad2d_matrix(want)
    # a decision that flips at an ambiguous pixel moves a Gaussian's gradient by
    # at most its own terms there (want["amb_abs"])
    for cols in (slice(0, 2), slice(2, 5), slice(5, 6), slice(6, 9)):
        w = W9[a, cols]
        good, worst = pu.close_bound(g2[a, cols], w, 1e-3, 1e-2 * np.abs(w).max(), want["amb_abs"][a, cols])
        assert good, (cols, worst)
    assert np.all(g2[:, 9:] == 0)


def test_project_backward_matches_oracle():
    st = _stage_inputs("tiny", frozen_frac=0.25, seed=3)
    n = st["P"].shape[0]
    g = np.random.default_rng(4)
    # raster gradients for every Gaussian, given to both sides identically
    g2 = pu.f32(g.normal(0, 1e-3, (n, 12)))
    g2[:, 9:] = 0
    grads2d = dict(d_mean2d=g2[:, 0:2], d_conic=g2[:, 2:5], d_opacity=g2[:, 5], d_rgb=g2[:, 6:9])
    act = np.nonzero(st["frozen"] == 0)[0].astype(np.int32)
    want = oracle.project_bwd(st["P"], st["ocam"], grads2d, st["frozen"])
    Pt = torch.from_numpy(pu.pack64(st["P"])).to(DEV)
    spl = torch.zeros((n, 12), device=DEV)
    lib.gs_project(Pt, n, 3, st["gcam"], spl)
    g2t = torch.from_numpy(g2.astype(np.float32)).to(DEV)
    G = torch.full((n, 64), 7.0, device=DEV)
    actt = torch.from_numpy(act).to(DEV)
    nact = torch.tensor([len(act)], dtype=torch.int32, device=DEV)
    ax = torch.zeros(n, device=DEV)
    ar = torch.zeros(n, device=DEV)
    cn = torch.zeros(n, dtype=torch.int32, device=DEV)
    lib.gs_project_bwd(Pt, n, 3, st["gcam"], spl, actt, nact, g2t, G, ax, ar, cn)
    torch.cuda.synchronize()
    G = G.cpu().numpy()
    g2_after = g2t.cpu().numpy()
    vis_gpu = spl.cpu().numpy()[:, 10].view(np.int32) > 0
    proj = oracle.project(st["P"], st["ocam"])
    safe = proj["margin"] > pu.PROJ_MARGIN
    fr = st["frozen"] == 1
    assert np.all(G[fr] == 7.0), "rows of frozen Gaussians are not touched"
    a = ~fr & safe
    assert np.all(G[a & ~vis_gpu][:, :] == 0)
    groups = [slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11), slice(11, 14), slice(14, 59)]
    av = a & vis_gpu
    for sl in groups:
        w = want["G"][av, sl]
        good, worst = pu.close(G[av, sl], w, 1e-3, 1e-2 * np.abs(w).max())
        assert good, (sl, worst)
    assert np.all(G[a, 59:] == 0)
    # raster gradients of processed Gaussians are consumed (zeroed)
    assert np.all(g2_after[av] == 0) and np.array_equal(g2_after[fr], g2[fr].astype(np.float32))
    # freeze statistics
    ax, ar, cn = ax.cpu().numpy(), ar.cpu().numpy(), cn.cpu().numpy()
    assert np.array_equal(cn[a], av[a].astype(np.int32))
    assert np.allclose(ax[av], want["xyz_norm"][av], rtol=1e-5, atol=1e-12)
    assert np.allclose(ar[av], want["rgb_norm"][av], rtol=1e-5, atol=1e-12)


# ----------------------------------------------------------------------------- A7 freeze update (bit-exact)


@pytest.mark.parametrize("n", [0, 1, 1000, 1024, 4099, 200003])
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_freeze_update_bit_exact(n, mode):
    g = np.random.default_rng(n + 31 * mode)
    acc_x = (g.exponential(3e-5, n) * g.integers(0, 4, n)).astype(np.float32)
    acc_r = (g.exponential(1e-4, n) * g.integers(0, 4, n)).astype(np.float32)
    cnt = g.integers(0, 4, n).astype(np.int32)
    frozen = (g.uniform(0, 1, n) < 0.2).astype(np.uint8)
    ex, er = np.float32(4e-5), np.float32(1.1e-4)
    t = [torch.from_numpy(a.copy()).to(DEV) for a in (acc_x, acc_r, cnt, frozen)]
    act = torch.full((max(n, 1),), -1, dtype=torch.int32, device=DEV)
    na = torch.zeros(1, dtype=torch.int32, device=DEV)
    ws = torch.zeros(lib.gs_freeze_workspace_bytes(n), dtype=torch.uint8, device=DEV)
    lib.gs_freeze_update(n, *t, float(ex), float(er), mode, act, na, ws)
    want_act = oracle.freeze_update(acc_x, acc_r, cnt, frozen, ex, er, mode)
    k = int(na.item())
    assert k == len(want_act)
    assert np.array_equal(act.cpu().numpy()[:k], want_act)
    assert np.array_equal(t[3].cpu().numpy(), frozen)
    for got, want in zip(t[:3], (acc_x, acc_r, cnt)):  # zeroed by the oracle too, except in mode 3
        assert np.array_equal(got.cpu().numpy(), want)


# ----------------------------------------------------------------------------- A8 masked Adam


def test_adam_masked_matches_oracle_and_skips_frozen():
    """Both sides get the same float32 inputs (parameters, moments, gradients,
    rates, betas); the tolerance is relative to the magnitude of the terms each
    update adds, since m = b1 m + (1 - b1) g may cancel."""
    g = np.random.default_rng(8)
    n = 3001
    P = g.normal(size=(n, 59)).astype(np.float32)
    M = g.normal(0, 1e-3, (n, 59)).astype(np.float32)
    V = g.uniform(0, 1e-5, (n, 59)).astype(np.float32)
    G = g.normal(0, 1e-3, (n, 59)).astype(np.float32)
    frozen = (g.uniform(0, 1, n) < 0.4).astype(np.uint8)
    act = np.nonzero(frozen == 0)[0].astype(np.int32)
    lr = [float(np.float32(x)) for x in (1.6e-4 * 4.4, 5e-3, 1e-3, 0.025, 2.5e-3, 1.25e-4)]
    b1, b2, eps = float(np.float32(0.9)), float(np.float32(0.999)), float(np.float32(1e-15))
    step = 17
    Pt, Mt, Vt, Gt = (torch.from_numpy(pu.pack64(a)).to(DEV) for a in (P, M, V, G))
    lib.gs_adam_masked(Pt, Gt, Mt, Vt, n, torch.from_numpy(act).to(DEV),
                       torch.tensor([len(act)], dtype=torch.int32, device=DEV), lr, b1, b2, eps, step)
    torch.cuda.synchronize()
    Po, Mo, Vo = (P.astype(np.float64), M.astype(np.float64), V.astype(np.float64))
    Gd = G.astype(np.float64)
    oracle.adam(Po, Gd, Mo, Vo, frozen, np.array(lr), step, b1=b1, b2=b2, eps=eps)
    Pg, Mg, Vg = (t.cpu().numpy()[:, :59] for t in (Pt, Mt, Vt))
    fr = frozen == 1
    assert np.array_equal(Pg[fr], P[fr]) and np.array_equal(Mg[fr], M[fr]) and np.array_equal(Vg[fr], V[fr])
    a = ~fr
    m_scale = b1 * np.abs(M[a]) + (1 - b1) * np.abs(Gd[a])
    v_scale = b2 * V[a] + (1 - b2) * Gd[a] ** 2
    assert np.all(np.abs(Mg[a] - Mo[a]) <= 1e-5 * m_scale)
    assert np.all(np.abs(Vg[a] - Vo[a]) <= 1e-5 * v_scale)
    # the step taken: |dp| <= lr m_hat / sqrt(v_hat); compare within 1e-4 of that bound
    group = np.array([0] * 3 + [1] * 3 + [2] * 4 + [3] + [4] * 3 + [5] * 45)
    bc1, bc2 = 1 - b1 ** step, 1 - b2 ** step
    bound = np.array(lr)[group] * (m_scale / bc1) / (np.sqrt(Vo[a] / bc2) + eps)
    spacing = np.spacing(np.abs(P[a]).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(Pg[a] - Po[a]) <= 1e-4 * bound + 2 * spacing)
    assert np.all(Pt.cpu().numpy()[:, 59:] == 0)


# ----------------------------------------------------------------------------- A9 PSNR


def test_psnr_matches_oracle():
    g = np.random.default_rng(9)
    S, H, W = 4, 57, 91
    gt = pu.f32(g.uniform(0, 1, (S, 3, H, W)))
    img = pu.f32(gt + g.normal(0, 0.05, gt.shape))
    img[1] = gt[1]  # identical: 100 dB floor
    img[2] += 0.7  # mostly clamped
    want = oracle.psnr(img, gt)
    it = torch.from_numpy(img.astype(np.float32)).to(DEV)
    gtt = torch.from_numpy(gt.astype(np.float32)).to(DEV)
    ws = torch.zeros(lib.gs_psnr_workspace_bytes(S, H, W), dtype=torch.uint8, device=DEV)
    out = torch.zeros(S, device=DEV)
    lib.gs_psnr(it, gtt, S, H, W, ws, out)
    got = out.cpu().numpy()
    assert got[1] == pytest.approx(100.0, abs=1e-4)
    assert np.allclose(got, want, rtol=1e-5, atol=1e-4)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_every_launch_shape_gives_the_same_result(tile):
    """Pixels per thread and batch size change only the launch shape: the
    forward is bit-identical and the backward equal up to atomic reordering."""
    st = _stage_inputs("ragged" if tile != 16 else "surface", tile)
    n = st["P"].shape[0]
    gcam = st["gcam"]
    vals = torch.from_numpy(st["vals"].view(np.int32).copy()).to(DEV)
    ranges = torch.from_numpy(st["ranges"].view(np.int32).copy()).to(DEV)
    H, W = gcam.height, gcam.width
    dlt = torch.from_numpy(st["dl"].astype(np.float32)).to(DEV)
    fr = torch.from_numpy(st["frozen"]).to(DEV)
    ref = None
    for ppt in (1, 2, 4) if tile >= 16 else (1, 2):
        for batch in (32, 64, 128, 256):
            cfg = lib.raster_config(ppt, batch)
            img = torch.zeros((3, H, W), device=DEV)
            tf = torch.zeros((H, W), device=DEV)
            nl = torch.zeros((H, W), dtype=torch.int32, device=DEV)
            lib.gs_render_fwd_cfg(st["spl"], vals, ranges, gcam, cfg, img, tf, nl)
            g2 = torch.zeros((n, 12), device=DEV)
            lib.gs_raster_bwd_cfg(st["spl"], vals, ranges, gcam, cfg, tf, nl, dlt, fr, g2)
            torch.cuda.synchronize()
            out = (img.cpu().numpy(), tf.cpu().numpy(), nl.cpu().numpy(), g2.cpu().numpy())
            if ref is None:
                ref = out
                continue
            assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
            assert np.array_equal(out[2], ref[2])
            good, worst = pu.close(out[3], ref[3], 1e-4, 1e-3 * np.abs(ref[3]).max())
            assert good, (ppt, batch, worst)


def test_four_pixels_per_thread_needs_a_16_pixel_tile():
    st = _stage_inputs("ragged", 8)
    gcam = st["gcam"]
    vals = torch.from_numpy(st["vals"].view(np.int32).copy()).to(DEV)
    ranges = torch.from_numpy(st["ranges"].view(np.int32).copy()).to(DEV)
    H, W = gcam.height, gcam.width
    img, tf = torch.zeros((3, H, W), device=DEV), torch.zeros((H, W), device=DEV)
    nl = torch.zeros((H, W), dtype=torch.int32, device=DEV)
    with pytest.raises(lib.GsError):
        lib.gs_render_fwd_cfg(st["spl"], vals, ranges, gcam, lib.raster_config(4, 64), img, tf, nl)
