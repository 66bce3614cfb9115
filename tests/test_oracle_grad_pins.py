"""Pins of the FP64 oracle's backward path, loss, Adam, freeze rule and PSNR:
central finite differences, closed forms and invariants. CPU only."""
import math

import numpy as np
import pytest

from paper_2504_06716_gb300 import synth


def _small_scene(orc, n=8, W=24, H=20, tile=8, seed=7, dilation=0.3, bg=(0.05, 0.1, 0.15)):
    g = np.random.default_rng(seed)
    P = np.zeros((n, 59))
    P[:, 0:3] = g.uniform(-0.35, 0.35, (n, 3))
    P[:, 3:6] = g.normal(-1.6, 0.3, (n, 3))
    P[:, 6:10] = g.normal(size=(n, 4))
    P[:, 10] = g.uniform(-1.0, 1.5, n)
    P[:, 11:] = g.normal(0, 0.3, 48)
    cam = synth.pinhole(W, H, 60.0, (0.2, -3.0, 0.3))
    gt = g.uniform(0, 1, (3, H, W))
    return P, orc.make_cam(cam, tile=tile, dilation=dilation, bg=bg), gt


def test_gradients_match_central_differences_smooth(orc):
    """Analytic gradient of L (Eq. 3) through compositing (Eq. 2), SH colour and
    projection (Eq. 1) against central differences of the loss, all 59
    parameters of every Gaussian, with the cut-offs switched off."""
    P, cam, gt = _small_scene(orc)
    res = orc.loss_and_grad(P, cam, gt, smooth=True)
    G = res["G"]
    h = 1e-5
    fd = np.zeros_like(P)
    for i in range(P.shape[0]):
        for k in range(59):
            Pp, Pm = P.copy(), P.copy()
            Pp[i, k] += h
            Pm[i, k] -= h
            fd[i, k] = (orc.loss_only(Pp, cam, gt, smooth=True) - orc.loss_only(Pm, cam, gt, smooth=True)) / (2 * h)
    scale = np.abs(fd).max()
    err = np.abs(G - fd)
    assert np.all(err <= 1e-5 * np.abs(fd) + 1e-7 * scale), (err / (np.abs(fd) + 1e-7 * scale)).max()
    assert np.abs(G[:, 11:]).max() > 0 and np.abs(G[:, :11]).max() > 0


def test_gradients_match_central_differences_with_cutoffs(orc):
    """With the real cut-offs the loss is piecewise smooth. At test points whose
    per-pixel and per-Gaussian decisions do not change under the perturbation,
    central differences still hold."""
    P, cam, gt = _small_scene(orc, n=10, W=40, H=32, tile=16, seed=21)
    P[:, 3:6] -= 0.6
    res = orc.loss_and_grad(P, cam, gt)
    h = 1e-6
    checked = 0
    for i in range(P.shape[0]):
        for k in list(range(11)) + [11, 12, 13, 20, 40, 58]:
            Pp, Pm = P.copy(), P.copy()
            Pp[i, k] += h
            Pm[i, k] -= h
            fp, fm = orc.forward(Pp, cam), orc.forward(Pm, cam)
            same = (np.array_equal(fp["n_last"], fm["n_last"]) and np.array_equal(fp["vals"], fm["vals"])
                    and np.array_equal(fp["proj"]["radius"], fm["proj"]["radius"])
                    and np.array_equal(fp["image"] > cam.bg[0], fm["image"] > cam.bg[0]))
            if not same:
                continue
            lp = orc.loss(fp["image"], gt, grad=False)[0]
            lm = orc.loss(fm["image"], gt, grad=False)[0]
            fd = (lp - lm) / (2 * h)
            assert res["G"][i, k] == pytest.approx(fd, rel=1e-4, abs=1e-9)
            checked += 1
    assert checked > 100


def test_gradients_at_the_clamped_screen_coordinate(orc):
    """The projection Jacobian takes x/z and y/z clamped to 1.3 times the
    half field of view, so beyond that limit the mean reaches the 2-D
    covariance only through 1/z: central differences of the loss see no
    dependence through the clamped coordinate. Two large anisotropic
    Gaussians whose centres lie past the limit (one in x, one in y) still
    cover pixels; the analytic gradient of every parameter must match."""
    W, H, f = 40, 32, 50.0
    cam = orc.make_cam(synth.Camera(W, H, f, f, W / 2.0, H / 2.0, np.eye(3), np.zeros(3), np.zeros(3)),
                       tile=8, dilation=0.3, bg=(0.05, 0.1, 0.15))
    g = np.random.default_rng(5)
    limx, limy = 1.3 * 0.5 * W / f, 1.3 * 0.5 * H / f
    P = np.zeros((2, 59))
    P[0, 0:3] = [(limx + 0.1234) * 3.0, 0.1, 3.0]
    P[1, 0:3] = [-0.2, -(limy + 0.1) * 3.4, 3.4]
    P[:, 3:6] = [[-0.3, -0.9, -0.6], [-1.0, -0.4, -0.7]]
    P[:, 6:10] = g.normal(size=(2, 4))
    P[:, 10] = [0.8, 0.5]
    P[:, 11:] = g.normal(0, 0.3, (2, 48))
    u, v = P[:, 0] / P[:, 2], P[:, 1] / P[:, 2]
    assert u[0] > limx and abs(v[0]) < limy and v[1] < -limy and abs(u[1]) < limx
    gt = g.uniform(0, 1, (3, H, W))
    res = orc.loss_and_grad(P, cam, gt, smooth=True)
    assert np.all(res["fwd"]["proj"]["radius"] > 0)
    G = res["G"]
    h = 1e-5
    fd = np.zeros_like(P)
    for i in range(2):
        for k in range(59):
            Pp, Pm = P.copy(), P.copy()
            Pp[i, k] += h
            Pm[i, k] -= h
            fd[i, k] = (orc.loss_only(Pp, cam, gt, smooth=True) - orc.loss_only(Pm, cam, gt, smooth=True)) / (2 * h)
    scale = np.abs(fd).max()
    err = np.abs(G - fd)
    assert np.all(err <= 1e-5 * np.abs(fd) + 1e-7 * scale), (err / (np.abs(fd) + 1e-7 * scale)).max()
    assert np.abs(G[:, 0:3]).min() > 1e-4 * scale


def test_frozen_rows_get_no_gradient_and_active_rows_are_unchanged(orc):
    """Sec. 3.2.4: frozen Gaussians skip the gradient; unfrozen rows are exactly
    what the unmasked backward gives."""
    P, cam, gt = _small_scene(orc, n=30, W=48, H=40, tile=16, seed=2)
    frozen = np.zeros(30, np.uint8)
    frozen[::3] = 1
    full = orc.loss_and_grad(P, cam, gt)
    masked = orc.loss_and_grad(P, cam, gt, frozen=frozen)
    act = frozen == 0
    assert np.array_equal(masked["G"][act], full["G"][act])
    assert np.all(masked["G"][~act] == 0)
    assert np.all(masked["xyz_norm"][~act] == 0) and np.all(masked["rgb_norm"][~act] == 0)
    assert np.abs(full["G"][~act]).max() > 0


def test_freeze_statistics_definitions(orc):
    """xyz_norm is |dL/d mean2d| scaled by (W/2, H/2); rgb_norm is |dL/d k_0|."""
    P, cam, gt = _small_scene(orc, n=12, W=40, H=30, tile=8, seed=4)
    r = orc.loss_and_grad(P, cam, gt)
    dm = r["grads2d"]["d_mean2d"]
    want = np.hypot(dm[:, 0] * cam.width / 2, dm[:, 1] * cam.height / 2)
    assert np.allclose(r["xyz_norm"], want, rtol=1e-14, atol=0)
    assert np.allclose(r["rgb_norm"], np.linalg.norm(r["G"][:, 11:14], axis=1), rtol=1e-14, atol=0)


# ----------------------------------------------------------------------------- loss


def test_loss_identical_images_is_zero_with_zero_gradient(orc):
    x = np.random.default_rng(0).uniform(0, 1, (3, 17, 23))
    L, g = orc.loss(x, x)
    assert abs(L) < 1e-15
    assert np.abs(g).max() < 1e-15


def test_loss_single_pixel_closed_form(orc):
    """For a 1x1 image only the window centre w0 = g(0)^2 / (sum_k g(k))^2 lies
    inside: mu = w0 x, sigma_x^2 = w0 x^2 - (w0 x)^2, sigma_xy = w0 x y - w0^2 x y."""
    x = np.array([0.8, 0.3, 0.55]).reshape(3, 1, 1)
    y = np.array([0.2, 0.35, 0.5]).reshape(3, 1, 1)
    gk = np.exp(-np.arange(-5, 6) ** 2 / (2 * 1.5 ** 2))
    w0 = 1.0 / gk.sum() ** 2
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    mx, my = w0 * x, w0 * y
    sx, sy, sxy = w0 * x * x - mx * mx, w0 * y * y - my * my, w0 * x * y - mx * my
    ssim = ((2 * mx * my + C1) * (2 * sxy + C2) / ((mx ** 2 + my ** 2 + C1) * (sx + sy + C2))).mean()
    want = 0.8 * np.abs(x - y).mean() + 0.2 * (1 - ssim)
    assert orc.loss(x, y, grad=False)[0] == pytest.approx(want, rel=1e-14)


def test_loss_equals_ssim_from_library_convolutions(orc):
    """Eq. 3 against an independent statement: the 11x11 Gaussian window
    (sigma 1.5, normalised) applied with scipy's 2-D convolution (zero fill
    outside the image), SSIM = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 +
    C1)(sx + sy + C2)) with C1 = 0.01^2, C2 = 0.03^2, averaged over the three
    channels; L = 0.8 mean|x - y| + 0.2 (1 - SSIM)."""
    from scipy.signal import convolve2d

    g = np.random.default_rng(4)
    H, W = 23, 31
    x = g.uniform(0, 1, (3, H, W))
    y = np.clip(x + g.normal(0, 0.2, (3, H, W)), 0, 1)
    t = np.exp(-((np.arange(11) - 5.0) ** 2) / (2 * 1.5 ** 2))
    t /= t.sum()
    w = np.outer(t, t)

    def filt(a):
        return convolve2d(a, w, mode="same", boundary="fill", fillvalue=0.0)

    C1, C2 = 0.01 ** 2, 0.03 ** 2
    ssim = []
    for c in range(3):
        mx, my = filt(x[c]), filt(y[c])
        sx, sy, sxy = filt(x[c] ** 2) - mx ** 2, filt(y[c] ** 2) - my ** 2, filt(x[c] * y[c]) - mx * my
        ssim.append((2 * mx * my + C1) * (2 * sxy + C2) / ((mx ** 2 + my ** 2 + C1) * (sx + sy + C2)))
    want = 0.8 * np.abs(x - y).mean() + 0.2 * (1.0 - np.mean(ssim))
    got = orc.loss(x, y, grad=False)[0]
    assert got == pytest.approx(want, rel=1e-12, abs=1e-14)
    assert orc.loss(x, y, lam=0.5, grad=False)[0] == pytest.approx(
        0.5 * np.abs(x - y).mean() + 0.5 * (1.0 - np.mean(ssim)), rel=1e-12)


def test_loss_is_symmetric(orc):
    g = np.random.default_rng(1)
    x, y = g.uniform(0, 1, (3, 19, 14)), g.uniform(0, 1, (3, 19, 14))
    assert orc.loss(x, y, grad=False)[0] == pytest.approx(orc.loss(y, x, grad=False)[0], rel=1e-14)


def test_loss_gradient_by_central_differences(orc):
    g = np.random.default_rng(3)
    x, y = g.uniform(0, 1, (3, 13, 16)), g.uniform(0, 1, (3, 13, 16))
    _, grad = orc.loss(x, y)
    h = 1e-6
    for _ in range(40):
        c, i, j = g.integers(3), g.integers(13), g.integers(16)
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = (orc.loss(xp, y, grad=False)[0] - orc.loss(xm, y, grad=False)[0]) / (2 * h)
        assert grad[c, i, j] == pytest.approx(fd, rel=1e-5, abs=1e-11)


def test_loss_windows_partition_the_loss(orc):
    """lambda + the window shares over any partition of the image = Eq. 3."""
    g = np.random.default_rng(4)
    x, y = g.uniform(0, 1, (3, 23, 31)), g.uniform(0, 1, (3, 23, 31))
    total = orc.loss(x, y, grad=False)[0]
    xs, ys = [0, 7, 8, 20, 31], [0, 5, 17, 23]
    parts = sum(orc.loss_window(x, y, xs[a], ys[b], xs[a + 1], ys[b + 1])
                for a in range(len(xs) - 1) for b in range(len(ys) - 1))
    assert 0.2 + parts == pytest.approx(total, rel=1e-13)


def test_loss_window_captures_a_local_change(orc):
    """A change confined to a region moves the loss exactly as much as the
    share of the window 5 pixels around that region."""
    g = np.random.default_rng(5)
    x, y = g.uniform(0, 1, (3, 40, 50)), g.uniform(0, 1, (3, 40, 50))
    x2 = x.copy()
    x2[:, 12:19, 30:36] += g.normal(0, 0.1, (3, 7, 6))
    d_full = orc.loss(x2, y, grad=False)[0] - orc.loss(x, y, grad=False)[0]
    d_win = orc.loss_window(x2, y, 25, 7, 41, 24) - orc.loss_window(x, y, 25, 7, 41, 24)
    assert d_win == pytest.approx(d_full, rel=1e-9, abs=1e-15)
    d_small = orc.loss_window(x2, y, 26, 8, 40, 23) - orc.loss_window(x, y, 26, 8, 40, 23)
    assert abs(d_small - d_full) > 1e-9  # one pixel less is not enough


# ----------------------------------------------------------------------------- Adam


def test_adam_first_steps_closed_form(orc):
    """Step 1: m_hat = g, v_hat = g^2, so p moves by lr * sign(g). Step 2 with
    gradient g2: m = 0.09 g + 0.1 g2 over 1 - 0.81, v = 0.000999 g^2 + 0.001 g2^2
    over 1 - 0.998001."""
    n = 4
    rng = np.random.default_rng(0)
    P = rng.normal(size=(n, 59))
    P0 = P.copy()
    M, V = np.zeros((n, 59)), np.zeros((n, 59))
    lr = np.array([1e-3, 2e-3, 3e-3, 4e-3, 5e-3, 6e-3])
    g1 = rng.normal(size=(n, 59))
    g1[1, 5] = 0.0
    orc.adam(P, g1, M, V, None, lr, step=1, eps=1e-15)
    group = np.array([0] * 3 + [1] * 3 + [2] * 4 + [3] + [4] * 3 + [5] * 45)
    assert np.allclose(P, P0 - lr[group] * np.sign(g1), rtol=0, atol=1e-15)
    assert P[1, 5] == P0[1, 5]
    g2 = rng.normal(size=(n, 59))
    P1 = P.copy()
    orc.adam(P, g2, M, V, None, lr, step=2, eps=1e-15)
    m = (0.9 * 0.1 * g1 + 0.1 * g2) / (1 - 0.81)
    v = (0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2) / (1 - 0.999 ** 2)
    assert np.allclose(P, P1 - lr[group] * m / (np.sqrt(v) + 1e-15), rtol=1e-13, atol=1e-16)


def test_adam_matches_torch_adam_over_several_steps(orc):
    """The oracle's Adam (Sec. 3.2.4's optimiser, vanilla 3DGS settings)
    against torch.optim.Adam in float64 with the six parameter groups as
    separate groups: five steps of random gradients, nothing frozen."""
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(17)
    n = 7
    P0 = g.normal(size=(n, 59))
    groups = [(0, 3), (3, 6), (6, 10), (10, 11), (11, 14), (14, 59)]
    lr = np.array([1.6e-4, 5e-3, 1e-3, 2.5e-2, 2.5e-3, 1.25e-4])
    b1, b2, eps = 0.9, 0.999, 1e-15
    tp = [torch.tensor(P0[:, a:b], dtype=torch.float64, requires_grad=True) for a, b in groups]
    opt = torch.optim.Adam([dict(params=[t], lr=float(r)) for t, r in zip(tp, lr)], betas=(b1, b2), eps=eps,
                           foreach=False)
    P, M, V = P0.copy(), np.zeros_like(P0), np.zeros_like(P0)
    for step in range(1, 6):
        G = g.normal(size=(n, 59)) * 10.0 ** g.uniform(-6, 0, (n, 59))
        for t, (a, b) in zip(tp, groups):
            t.grad = torch.tensor(G[:, a:b], dtype=torch.float64)
        opt.step()
        orc.adam(P, G, M, V, None, lr, step=step, b1=b1, b2=b2, eps=eps)
        want = np.concatenate([t.detach().numpy() for t in tp], axis=1)
        assert np.allclose(P, want, rtol=1e-12, atol=1e-15)


def test_adam_leaves_frozen_rows_bit_unchanged(orc):
    rng = np.random.default_rng(1)
    P, M, V = rng.normal(size=(6, 59)), rng.normal(size=(6, 59)), rng.uniform(0, 1, (6, 59))
    G = rng.normal(size=(6, 59))
    frozen = np.array([1, 0, 1, 0, 0, 1], np.uint8)
    P0, M0, V0 = P.copy(), M.copy(), V.copy()
    orc.adam(P, G, M, V, frozen, np.full(6, 1e-2), step=7)
    f = frozen == 1
    assert np.array_equal(P[f], P0[f]) and np.array_equal(M[f], M0[f]) and np.array_equal(V[f], V0[f])
    assert not np.array_equal(P[~f], P0[~f])


# ----------------------------------------------------------------------------- freeze rule


def test_freeze_update_hand_example(orc):
    """Eqs. 4-6 with eps_xyz = 1.0, eps_rgb = 2.0 on averaged statistics; strict
    comparisons, both conditions required, cnt = 0 never freezes, the map is
    sticky until a reset."""
    acc_x = np.array([0.5, 3.0, 0.5, 3.0, 0.0, 2.0, 0.9], np.float32)
    acc_r = np.array([1.0, 1.0, 5.0, 9.0, 0.0, 3.9, 1.0], np.float32)
    cnt = np.array([1, 2, 1, 1, 0, 2, 1], np.int32)
    frozen = np.array([0, 0, 0, 1, 0, 0, 0], np.uint8)
    # averages: x (0.5, 1.5, 0.5, 3, -, 1.0, 0.9), rgb (1, 0.5, 5, 9, -, 1.95, 1)
    act = orc.freeze_update(acc_x, acc_r, cnt, frozen, 1.0, 2.0, 0)
    assert frozen.tolist() == [1, 0, 0, 1, 0, 0, 1]
    assert act.tolist() == [1, 2, 4, 5]
    assert not acc_x.any() and not acc_r.any() and not cnt.any()
    act = orc.freeze_update(acc_x, acc_r, cnt, frozen, 1.0, 2.0, 2)  # clear: map kept
    assert frozen.tolist() == [1, 0, 0, 1, 0, 0, 1] and act.tolist() == [1, 2, 4, 5]
    act = orc.freeze_update(acc_x, acc_r, cnt, frozen, 1.0, 2.0, 1)  # reset
    assert not frozen.any() and act.tolist() == list(range(7))
    frozen[[0, 6]] = 1
    acc_x[:] = 0.25
    cnt[:] = 1
    act = orc.freeze_update(acc_x, acc_r, cnt, frozen, 1.0, 2.0, 3)  # list only: map and statistics kept
    assert act.tolist() == [1, 2, 3, 4, 5] and frozen.tolist() == [1, 0, 0, 0, 0, 0, 1]
    assert acc_x.tolist() == [0.25] * 7 and cnt.tolist() == [1] * 7


# ----------------------------------------------------------------------------- PSNR


def test_psnr_special_cases(orc):
    g = np.random.default_rng(0)
    gt = g.uniform(0, 1, (3, 3, 8, 9))
    img = gt.copy()
    img[1] = np.clip(gt[1] + 0.1, None, None)
    img[2] = gt[2] + 2.0  # clamps to 1
    p = orc.psnr(img, gt)
    assert p[0] == pytest.approx(100.0)
    # uniform error delta, values kept inside [0, 1]
    gt2 = g.uniform(0.2, 0.8, (1, 3, 5, 5))
    assert orc.psnr(gt2 + 0.05, gt2)[0] == pytest.approx(-20 * math.log10(0.05), rel=1e-12)
    assert p[2] == pytest.approx(10 * math.log10(1 / np.mean((1 - gt[2]) ** 2)), rel=1e-12)
