"""Pins of the FP64 oracle's forward path against facts fixed outside the oracle:
closed forms, quadrature, brute force and invariants. CPU only."""
import math

import numpy as np
import pytest

from paper_2504_06716_gb300 import synth


def _cam_on_axis(W=64, H=48, f=80.0, tile=16, dilation=0.0, bg=(0, 0, 0), orc=None):
    """Camera at the origin looking down +z (identity rotation)."""
    cam = synth.Camera(W, H, f, f, W / 2.0, H / 2.0, np.eye(3), np.zeros(3), np.zeros(3))
    return orc.make_cam(cam, tile=tile, dilation=dilation, bg=bg)


def _gauss(mean, log_s, quat=(1, 0, 0, 0), logit=0.0, dc=(0.0, 0.0, 0.0)):
    p = np.zeros(59)
    p[0:3] = mean
    p[3:6] = log_s
    p[6:10] = quat
    p[10] = logit
    p[11:14] = dc
    return p


# ----------------------------------------------------------------------------- SH


def test_sh_orthonormal_by_quadrature(orc):
    """The 16 real SH functions are orthonormal on the sphere (Gauss-Legendre in
    cos(theta) x uniform in phi; exact for these polynomial degrees)."""
    zs, wz = np.polynomial.legendre.leggauss(12)
    nphi = 24
    G = np.zeros((16, 16))
    for z, w in zip(zs, wz):
        s = math.sqrt(1 - z * z)
        for k in range(nphi):
            phi = 2 * math.pi * k / nphi
            Y = orc.sh_basis([s * math.cos(phi), s * math.sin(phi), z])
            G += w * (2 * math.pi / nphi) * np.outer(Y, Y)
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_basis_equals_library_spherical_harmonics(orc):
    """The real basis against scipy's complex spherical harmonics (which
    carry the Condon-Shortley phase): coefficient l^2 + l + m is
    sqrt(2) Re Y_l^m for m > 0, sqrt(2) Im Y_l^|m| for m < 0 and Y_l^0 for
    m = 0, at the polar angle of z and the azimuth of (x, y)."""
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    g = np.random.default_rng(8)
    for _ in range(50):
        d = g.normal(size=3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        want = []
        for l in range(4):
            for m in range(-l, l + 1):
                y = complex(sp.sph_harm_y(l, abs(m), theta, phi))
                want.append(math.sqrt(2) * y.real if m > 0 else math.sqrt(2) * y.imag if m < 0 else y.real)
        assert np.allclose(orc.sh_basis(d), want, rtol=1e-12, atol=1e-13)


def test_sh_band0_constant_and_band1_directions(orc):
    d = np.array([0.36, -0.48, 0.8])
    Y = orc.sh_basis(d)
    assert Y[0] == pytest.approx(1.0 / (2.0 * math.sqrt(math.pi)), abs=1e-15)
    # band 1 is sqrt(3/(4 pi)) times (-y, z, -x) with the Condon-Shortley phase
    c1 = math.sqrt(3.0 / (4.0 * math.pi))
    assert np.allclose(Y[1:4], c1 * np.array([-d[1], d[2], -d[0]]), atol=1e-15)
    # addition theorem: sum_m Y_lm(d)^2 = (2l+1)/(4 pi) for every band
    for l in range(4):
        assert np.sum(Y[l * l:(l + 1) * (l + 1)] ** 2) == pytest.approx((2 * l + 1) / (4 * math.pi), rel=1e-12)


def test_sh_gradient_by_finite_differences(orc):
    rng = np.random.default_rng(5)
    for _ in range(5):
        d = rng.normal(size=3)
        dY = orc.sh_basis_grad(d)
        h = 1e-6
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            fd = (orc.sh_basis(d + e) - orc.sh_basis(d - e)) / (2 * h)
            assert np.allclose(dY[:, a], fd, atol=1e-8)


# ----------------------------------------------------------------------------- closed forms


@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.2, 0.5, 0.9)])
def test_single_isotropic_gaussian_closed_form(orc, bg):
    """One isotropic Gaussian on the optical axis at depth z with scale s and no
    dilation images as C(u, v) = c a + (1 - a) bg with
    a = min(0.99, o exp(-((u-cx)^2 + (v-cy)^2) / (2 (f s / z)^2))) wherever
    a >= 1/255 and the pixel's tile lies within ceil(3 f s / z) of the centre."""
    W, H, f, z, s, tile = 64, 48, 80.0, 4.0, 0.21, 16  # 3 sigma = 12.6: off the ceil boundary
    cam = _cam_on_axis(W, H, f, tile, 0.0, bg, orc)
    dc = np.array([0.7, -0.3, 0.1])
    logit = 1.3
    P = _gauss([0, 0, z], [math.log(s)] * 3, quat=(0.3, 0.5, -0.2, 0.7), logit=logit, dc=dc)[None]
    f_ = orc.forward(P, cam, sh_degree=0)
    o = 1 / (1 + math.exp(-logit))
    c = np.maximum(dc / (2 * math.sqrt(math.pi)) + 0.5, 0)
    sig = f * s / z
    r = math.ceil(3 * sig)
    u, v = np.meshgrid(np.arange(W), np.arange(H))
    a = np.minimum(0.99, o * np.exp(-((u - W / 2) ** 2 + (v - H / 2) ** 2) / (2 * sig * sig)))
    tx0, tx1 = math.floor((W / 2 - r) / tile), math.floor((W / 2 + r) / tile)
    ty0, ty1 = math.floor((H / 2 - r) / tile), math.floor((H / 2 + r) / tile)
    inside = (u // tile >= tx0) & (u // tile <= tx1) & (v // tile >= ty0) & (v // tile <= ty1)
    a = np.where(inside & (a >= 1 / 255), a, 0.0)
    want = c[:, None, None] * a + (1 - a) * np.array(bg)[:, None, None]
    assert f_["proj"]["radius"][0] == r
    assert np.abs(f_["image"] - want).max() < 1e-12
    assert np.abs(f_["t_final"] - (1 - a)).max() < 1e-12


def test_two_gaussians_blend_front_to_back(orc):
    """Eq. 2 for two Gaussians on the axis: C = c1 a1 + c2 a2 (1 - a1) with the
    nearer one first, whatever their index order."""
    W, H, f = 32, 32, 60.0
    cam = _cam_on_axis(W, H, f, 16, 0.0, (0, 0, 0), orc)
    near = _gauss([0, 0, 3.0], [math.log(0.3)] * 3, logit=0.5, dc=(1.0, 0.0, 0.0))
    far = _gauss([0, 0, 5.0], [math.log(0.5)] * 3, logit=0.8, dc=(0.0, 1.0, 0.0))
    for order in ([far, near], [near, far]):
        f_ = orc.forward(np.stack(order), cam, sh_degree=0)
        u, v = W // 2, H // 2
        a1 = min(0.99, 1 / (1 + math.exp(-0.5)))
        a2 = min(0.99, 1 / (1 + math.exp(-0.8)))
        c1 = np.array([1.0, 0, 0]) / (2 * math.sqrt(math.pi)) + 0.5
        c2 = np.array([0, 1.0, 0]) / (2 * math.sqrt(math.pi)) + 0.5
        want = c1 * a1 + c2 * a2 * (1 - a1)
        assert np.allclose(f_["image"][:, v, u], want, atol=1e-12)


def test_equal_depths_blend_in_index_order(orc):
    """Splats at the same depth have equal sort keys; the stable sort keeps
    them in ascending Gaussian index, so with two copies of one Gaussian
    (different colours) the lower index is in front: C = c_lo a + c_hi a (1 - a),
    and every tile lists the lower index first."""
    W, H, f = 32, 32, 60.0
    cam = _cam_on_axis(W, H, f, 16, 0.0, (0, 0, 0), orc)
    red = _gauss([0, 0, 4.0], [math.log(0.4)] * 3, logit=0.3, dc=(1.0, 0.0, 0.0))
    blue = _gauss([0, 0, 4.0], [math.log(0.4)] * 3, logit=0.3, dc=(0.0, 0.0, 1.0))
    a = min(0.99, 1 / (1 + math.exp(-0.3)))
    cr = np.array([1.0, 0, 0]) / (2 * math.sqrt(math.pi)) + 0.5
    cb = np.array([0, 0, 1.0]) / (2 * math.sqrt(math.pi)) + 0.5
    for lo, hi, c_lo, c_hi in ((red, blue, cr, cb), (blue, red, cb, cr)):
        f_ = orc.forward(np.stack([lo, hi]), cam, sh_degree=0)
        assert f_["proj"]["depth"][0] == f_["proj"]["depth"][1]
        u, v = W // 2, H // 2
        assert np.allclose(f_["image"][:, v, u], c_lo * a + c_hi * a * (1 - a), atol=1e-12)
        rg = f_["ranges"]
        lists = [f_["vals"][s:e].tolist() for s, e in rg if e > s]
        assert lists and all(x == [0, 1] for x in lists)


def test_anisotropic_projection_closed_form(orc):
    """An axis-aligned Gaussian straight ahead of the camera projects to
    J S^2 J^T (+ dilation): variances (f s_x / z)^2 + d and (f s_y / z)^2 + d,
    no covariance; the conic is their inverse and the mean sits at (cx, cy)."""
    cam = _cam_on_axis(64, 64, 100.0, 16, 0.3, (0, 0, 0), orc)
    z, sx, sy = 5.0, 0.3, 0.1
    P = _gauss([0, 0, z], [math.log(sx), math.log(sy), math.log(0.2)])[None]
    pr = orc.project(P, cam, 0)
    vx, vy = (100 * sx / z) ** 2 + 0.3, (100 * sy / z) ** 2 + 0.3
    assert np.allclose(pr["conic"][0], [1 / vx, 0, 1 / vy], rtol=1e-12, atol=1e-15)
    assert np.allclose(pr["mean2d"][0], [32, 32], atol=1e-12)
    assert pr["depth"][0] == pytest.approx(z)
    assert pr["radius"][0] == math.ceil(3 * math.sqrt(max(vx, vy)))


def test_projected_covariance_from_library_rotation_and_numeric_jacobian(orc):
    """Eq. 1 against independent pieces: the rotation of the quaternion
    (w, x, y, z) from scipy's Rotation (scalar-last input), Sigma = R S^2 R^T,
    and the Jacobian of the pixel mapping mu -> (fx x_c / z_c + cx, fy y_c /
    z_c + cy) taken by central differences in world space; the 2-D
    covariance is J Sigma J^T + dilation I, its inverse the conic, the mean
    the mapping itself. Gaussians well inside the view (no clamping)."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    cam = synth.pinhole(96, 72, 60.0, (0.7, -3.5, 1.2))
    ocam = orc.make_cam(cam, tile=16, dilation=0.3)
    g = np.random.default_rng(12)
    n = 40
    P = np.zeros((n, 59))
    P[:, 0:3] = g.uniform(-0.4, 0.4, (n, 3))
    P[:, 3:6] = g.normal(-2.0, 0.4, (n, 3))
    P[:, 6:10] = g.normal(size=(n, 4))
    P[:, 10] = 1.0
    pr = orc.project(P, ocam, 0)
    R_c, t_c = np.asarray(cam.R), np.asarray(cam.t)

    def pix(mu):
        c = R_c @ mu + t_c
        return np.array([cam.fx * c[0] / c[2] + cam.cx, cam.fy * c[1] / c[2] + cam.cy])

    checked = 0
    for i in range(n):
        if pr["radius"][i] <= 0:
            continue
        q = P[i, 6:10]
        R = Rot.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sigma = R @ np.diag(np.exp(2 * P[i, 3:6])) @ R.T
        h = 1e-6
        J = np.stack([(pix(P[i, 0:3] + h * e) - pix(P[i, 0:3] - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        cov = J @ Sigma @ J.T + 0.3 * np.eye(2)
        conic = np.linalg.inv(cov)
        assert np.allclose(pr["conic"][i], [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=1e-7, atol=1e-12)
        assert np.allclose(pr["mean2d"][i], pix(P[i, 0:3]), rtol=1e-12, atol=1e-9)
        checked += 1
    assert checked > 30


def test_near_plane_and_offscreen_culling(orc):
    cam = _cam_on_axis(64, 64, 100.0, 16, 0.3, (0, 0, 0), orc)
    P = np.stack([
        _gauss([0, 0, 0.1], [-3] * 3),  # in front of the camera but inside the near plane
        _gauss([0, 0, -2.0], [-3] * 3),  # behind the camera
        _gauss([50, 0, 2.0], [-3] * 3),  # far off to the side: no tile touched
        _gauss([0, 0, 2.0], [-3] * 3),  # visible
    ])
    pr = orc.project(P, cam, 0)
    assert list(pr["radius"] > 0) == [False, False, False, True]
    assert list(pr["tiles_touched"]) == [0, 0, 0, pr["tiles_touched"][3]]


# ----------------------------------------------------------------------------- brute force


def _random_view(orc, n=300, W=72, H=56, tile=16, seed=3, bg=(0.1, 0.2, 0.3)):
    g = np.random.default_rng(seed)
    P = synth.gaussians_uniform(n, seed)
    P[:, 3:6] += 1.0  # larger splats so that lists overlap heavily
    P[:, 10] = g.uniform(-1, 3, n)
    cam = synth.pinhole(W, H, 60.0, (0.3, -0.4, 3.2))
    return P, orc.make_cam(cam, tile=tile, bg=bg)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_tiled_render_equals_brute_force(orc, tile):
    P, cam = _random_view(orc, tile=tile)
    f = orc.forward(P, cam)
    brute = orc.render_brute(f["proj"], cam)
    assert (f["proj"]["radius"] > 0).sum() > 100
    assert np.abs(f["image"] - brute).max() < 1e-12


SLACK = 3e-4  # the oracle lists splats whose alpha comes within this relative distance of the floor


def test_sort_lists_isotropic_closed_form(orc):
    """Isotropic splats (conic a = c = 1/s^2, b = 0): alpha = o exp(-r^2 / (2 s^2))
    reaches (1 - SLACK) / 255, the floor of Eq. 2 with the oracle's slack,
    within the distance R = s sqrt(2 ln(255 o / (1 - SLACK))) of the mean, so a
    tile of the 3-sigma rectangle lists the splat exactly when the pixel centre
    of the tile (inside the image) nearest to the mean lies within R. Each
    tile's list is in (float32 depth, index) order."""
    g = np.random.default_rng(21)
    n, W, H, tile = 700, 150, 93, 16
    mx = g.uniform(-25, W + 25, n)
    my = g.uniform(-25, H + 25, n)
    s = g.uniform(0.7, 14.0, n)
    o = np.exp(g.uniform(np.log(0.002), 0.0, n))
    o[:20] = (1.0 - SLACK) / 255.0 - 1e-6  # below the floor: listed nowhere
    rad = np.ceil(3 * s).astype(np.int32)
    depth = g.choice(np.array([1.0, 2.5, 4.0], np.float32), n)  # many equal depths: index breaks ties
    m32 = np.stack([mx, my], 1).astype(np.float32)
    inv = (1.0 / (s * s)).astype(np.float32)
    q32 = np.stack([inv, np.zeros(n, np.float32), inv], 1)
    o32 = o.astype(np.float32)
    vals, ranges = orc.sort(m32, q32, o32, rad, depth, W, H, tile)
    tx, ty = (W + tile - 1) // tile, (H + tile - 1) // tile
    M, S2, O = m32.astype(np.float64), 1.0 / q32[:, 0].astype(np.float64), o32.astype(np.float64)
    want, ambiguous = [], set()
    for i in range(n):
        x0 = max(int(np.floor((m32[i, 0] - rad[i]) / np.float32(tile))), 0)
        x1 = min(int(np.floor((m32[i, 0] + rad[i]) / np.float32(tile))), tx - 1)
        y0 = max(int(np.floor((m32[i, 1] - rad[i]) / np.float32(tile))), 0)
        y1 = min(int(np.floor((m32[i, 1] + rad[i]) / np.float32(tile))), ty - 1)
        if O[i] * 255.0 < 1.0 - SLACK:
            continue
        R2 = S2[i] * 2.0 * np.log(255.0 * O[i] / (1.0 - SLACK))
        for y in range(y0, y1 + 1):
            for x in range(x0, x1 + 1):
                nx = min(max(round(M[i, 0]), x * tile), min(x * tile + tile, W) - 1)
                ny = min(max(round(M[i, 1]), y * tile), min(y * tile + tile, H) - 1)
                d2 = (nx - M[i, 0]) ** 2 + (ny - M[i, 1]) ** 2
                if abs(d2 - R2) <= 1e-9 * R2:
                    ambiguous.add((y * tx + x, i))
                elif d2 <= R2:
                    want.append((y * tx + x, i))
    got = [(t, int(i)) for t in range(tx * ty) for i in vals[ranges[t, 0]:ranges[t, 1]]]
    assert set(got) - ambiguous == set(want) and len(want) > 500
    assert all(i >= 20 for _, i in got)
    for t in range(tx * ty):
        ids = vals[ranges[t, 0]:ranges[t, 1]].tolist()
        assert ids == sorted(ids, key=lambda i: (float(depth[i]), i))


def test_sort_lists_are_minimal(orc):
    """Every entry of a tile's list blends at some pixel of that tile, but for
    the slack band: on a scene whose rays never reach the transmittance floor
    (few, faint splats), each listed splat appears in the compositing trace of
    at least one pixel of the tile, except entries whose largest alpha over
    the tile's pixel centres lies in [(1 - SLACK) / 255, 1 / 255). Together
    with the untiled brute-force render (no contribution missing), this fixes
    the lists."""
    g = np.random.default_rng(5)
    P, cam = _random_view(orc, n=120, W=64, H=48, tile=16, seed=13)
    op = g.uniform(0.004, 0.3, P.shape[0])
    P[:, 10] = np.log(op / (1 - op))
    f = orc.forward(P, cam)
    vals, ranges = f["vals"], f["ranges"]
    tx = (cam.width + 15) // 16
    seen = set()
    for py in range(cam.height):
        for px in range(cam.width):
            pos, al, tr = orc.pixel_trace(f["proj"], vals, ranges, cam, px, py)
            assert len(tr) == 0 or tr[-1] * (1 - al[-1]) > 1e-3  # no ray near the floor
            t = (py // 16) * tx + px // 16
            seen.update((t, int(vals[ranges[t, 0] + p])) for p in pos)
    listed = {(t, int(i)) for t in range(len(ranges)) for i in vals[ranges[t, 0]:ranges[t, 1]]}
    assert len(listed) > 100 and seen <= listed
    pr = f["proj"]
    for t, i in listed - seen:  # the slack band only
        x0, y0 = (t % tx) * 16, (t // tx) * 16
        ys, xs = np.mgrid[y0:min(y0 + 16, cam.height), x0:min(x0 + 16, cam.width)]
        dx, dy = xs - pr["mean2d"][i, 0], ys - pr["mean2d"][i, 1]
        a, b, c = pr["conic"][i]
        amax = (pr["opacity"][i] * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy))).max()
        assert (1 - SLACK) / 255 <= amax < 1 / 255, (t, i, amax * 255)
    assert np.abs(f["image"] - orc.render_brute(f["proj"], cam)).max() < 1e-12


def test_transmittance_non_increasing_along_rays(orc):
    P, cam = _random_view(orc, n=600, seed=11)
    f = orc.forward(P, cam)
    checked = 0
    for py in range(0, cam.height, 5):
        for px in range(0, cam.width, 5):
            pos, al, tr = orc.pixel_trace(f["proj"], f["vals"], f["ranges"], cam, px, py)
            if len(al) == 0:
                continue
            checked += 1
            assert np.all(np.diff(tr) <= 0)
            assert np.all((al >= 1 / 255) & (al <= 0.99))
            assert tr[-1] * (1 - al[-1]) >= 1e-4
            assert f["t_final"][py, px] == pytest.approx(tr[-1] * (1 - al[-1]), rel=1e-12)
            assert f["n_last"][py, px] == pos[-1] + 1
    assert checked > 50


def test_early_termination_by_transmittance(orc):
    """A stack of Gaussians with alpha = 0.95 at the centre pixel: T runs
    1, 0.05, 0.0025, 1.25e-4; the fourth layer would take it to 6.25e-6 < 1e-4,
    so the ray stops before it and exactly three layers contribute."""
    cam = _cam_on_axis(32, 32, 60.0, 16, 0.0, (0, 0, 0), orc)
    logit = math.log(0.95 / 0.05)
    P = np.stack([_gauss([0, 0, 2.0 + 0.5 * k], [math.log(0.5)] * 3, logit=logit, dc=(k, 0, 0)) for k in range(5)])
    f = orc.forward(P, cam, sh_degree=0)
    pos, al, tr = orc.pixel_trace(f["proj"], f["vals"], f["ranges"], cam, 16, 16)
    assert np.allclose(al, [0.95] * 3, rtol=1e-12) and np.allclose(tr, [1.0, 0.05, 0.0025], rtol=1e-12)
    assert f["t_final"][16, 16] == pytest.approx(1.25e-4, rel=1e-9)
    c = (np.arange(3) / (2 * math.sqrt(math.pi)) + 0.5) * 0.95 * np.array([1.0, 0.05, 0.0025])
    assert f["image"][0, 16, 16] == pytest.approx(c.sum(), rel=1e-12)
