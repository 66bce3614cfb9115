"""Whole-step parity of the CUDA path with the oracle, and row-by-row parity
at the mid-size workload's full size (1M Gaussians, 1237x822, the launch
configuration bench.py times) on outputs the oracle can compute one by one."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2504_06716_gb300 import lib, pipeline, synth  # noqa: E402

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


def _nudge(P, ocam, tries=20):
    """Move Gaussians whose radius or tile rectangle sits within PROJ_MARGIN of
    a boundary slightly off it (their log-scales and means), so that the
    float32 and float64 projections take the same integer decisions."""
    P = P.copy()
    for _ in range(tries):
        pr = oracle.project(P, ocam)
        bad = pr["margin"] <= pu.PROJ_MARGIN
        if not bad.any():
            return pu.f32(P)
        P[bad, 3:6] += 3e-3
        P[bad, 0] += 1e-3
        P = pu.f32(P)
    raise AssertionError("could not move every Gaussian off a decision boundary")


# ----------------------------------------------------------------------------- one whole step, tiny workload


@pytest.mark.parametrize("cam_index", [0, 3, 6])
def test_full_step_matches_oracle(cam_index):
    """project -> sort -> render -> loss -> backward (frozen skipped) -> masked
    Adam on the 2,000-Gaussian workload, against the oracle's step on the same
    float32 inputs."""
    s = synth.tiny_scene()
    ocam, gcam = pu.cameras(s.cameras[cam_index])
    P = _nudge(pu.f32(s.init), ocam)
    gt = pu.f32(oracle.forward(pu.f32(s.gt), ocam)["image"])
    n = P.shape[0]
    frozen = (np.random.default_rng(cam_index).uniform(0, 1, n) < 0.3).astype(np.uint8)

    m = pipeline.Model(P)
    m.frozen.copy_(torch.from_numpy(frozen))
    m.freeze_update(0.0, 0.0, 2)
    view = m.make_view(gcam, m.measure_capacity([gcam]))
    gt_t = torch.from_numpy(gt.astype(np.float32)).to(DEV)
    lrs = [float(np.float32(x)) for x in pipeline.default_lrs(4.4)]
    m.rasterize(view)
    m.loss(view, gt_t)
    m.backward(view)
    G_gpu = m.G.cpu().numpy()[:, :59].copy()
    m.adam(lrs, b1=float(np.float32(0.9)), b2=float(np.float32(0.999)), eps=float(np.float32(1e-15)))
    torch.cuda.synchronize()
    assert lib.gs_get_device_error() == 0

    want = oracle.loss_and_grad(P, ocam, gt, frozen=frozen)
    img = view.image.cpu().numpy()
    amb = want["fwd"]["margin"] <= pu.E2E_PIXEL_MARGIN  # decisions float32 may take either way
    assert amb.mean() < 0.05
    good, worst = pu.close(img, want["fwd"]["image"], 1e-4, 1.0, np.broadcast_to(~amb, img.shape))
    assert good, worst
    assert float(view.loss.item()) == pytest.approx(want["loss"], rel=1e-4)

    # every active Gaussian is compared; a decision flipping at an ambiguous
    # pixel moves its gradient by at most its own terms there, carried
    # through the projection Jacobian
    rb = oracle.render_bwd(want["fwd"]["proj"], want["fwd"]["vals"], want["fwd"]["ranges"], ocam, want["dl_dimage"],
                           frozen, amb.astype(np.uint8))
    l1 = pu.l1_sign_bound(want["fwd"]["proj"], want["fwd"]["vals"], want["fwd"]["ranges"], ocam, want["fwd"]["image"],
                          gt, frozen)
    bound = pu.param_bound(P, ocam, rb["amb_abs"] + l1, frozen)
    fr = frozen == 1
    act = ~fr & (want["fwd"]["proj"]["radius"] > 0)
    for sl in [slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11), slice(11, 14), slice(14, 59)]:
        w = want["G"][act, sl]
        good, worst = pu.close_bound(G_gpu[act, sl], w, 1e-3, 1e-2 * np.abs(w).max(), bound[act, sl])
        assert good, (sl, worst)
    P_gpu = m.P.cpu().numpy()[:, :59]
    assert np.array_equal(P_gpu[fr], P[fr].astype(np.float32))
    Po = P.copy()
    M, V = np.zeros_like(Po), np.zeros_like(Po)
    oracle.adam(Po, want["G"], M, V, frozen, np.array(lrs), 1, b1=float(np.float32(0.9)),
                b2=float(np.float32(0.999)), eps=float(np.float32(1e-15)))
    # first Adam step moves each parameter by about lr * sign(g): compare the direction
    # and size where the gradient is clearly non-zero
    big = act[:, None] & (np.abs(want["G"]) > 1e-2 * np.abs(want["G"]).max(axis=0, keepdims=True)) & (bound == 0)
    assert np.allclose(P_gpu[big], Po[big], rtol=0, atol=1e-6 + 1e-3 * np.abs(Po[big]).max())


# ----------------------------------------------------------------------------- full size, sampled


@pytest.fixture(scope="module")
def mid():
    """The mid-size workload: 1M Gaussians on the surface mix, one 1237x822 view."""
    s = synth.surface_scene(1_000_000, 10, 200, 1237, 822)
    cam = s.cameras[s.train_views[5]]
    ocam, gcam = pu.cameras(cam)
    P = pu.f32(s.init)
    pr = oracle.project(P, ocam)
    rec = pu.records_from_oracle(pr)
    return dict(P=P, ocam=ocam, gcam=gcam, pr=pr, rec=rec, proj=pu.proj_from_records(rec))


def test_fullsize_project_sampled(mid):
    n = mid["P"].shape[0]
    Pt = torch.from_numpy(pu.pack64(mid["P"])).to(DEV)
    spl = torch.zeros((n, 12), device=DEV)
    lib.gs_project(Pt, n, 3, mid["gcam"], spl)
    got = spl.cpu().numpy()
    pr = mid["pr"]
    safe = pr["margin"] > pu.PROJ_MARGIN
    assert safe.mean() > 0.99
    rad = got[:, 10].view(np.int32)
    assert np.array_equal(rad[safe], pr["radius"][safe])
    assert np.array_equal(got[safe, 11].view(np.int32), pr["tiles_touched"][safe])
    vis = safe & (pr["radius"] > 0)
    assert np.abs(got[vis, 0:2] - pr["mean2d"][vis]).max() < 2e-3
    scale = np.maximum(np.abs(pr["conic"][vis, 0]), np.abs(pr["conic"][vis, 2]))[:, None]
    assert (np.abs(got[vis, 2:5] - pr["conic"][vis]) / scale).max() < 1e-4
    assert np.abs(got[vis, 6:9] - pr["rgb"][vis]).max() < 1e-5


@pytest.fixture(scope="module")
def mid_sorted(mid):
    n = mid["rec"].shape[0]
    cap = int(mid["rec"][:, 11].view(np.int32).astype(np.int64).sum()) + 4096
    spl = torch.from_numpy(mid["rec"]).to(DEV)
    ws = torch.zeros(lib.gs_sort_workspace_bytes(n, cap, mid["gcam"]), dtype=torch.uint8, device=DEV)
    vals = torch.zeros(cap, dtype=torch.int32, device=DEV)
    ranges = torch.zeros((mid["gcam"].tiles, 2), dtype=torch.int32, device=DEV)
    count = torch.zeros(1, dtype=torch.int64, device=DEV)
    lib.gs_sort(spl, n, mid["gcam"], ws, cap, vals, ranges, count)
    return dict(spl=spl, vals=vals, ranges=ranges, count=int(count.item()))


def test_fullsize_sort_matches_oracle(mid, mid_sorted):
    want_vals, want_ranges = oracle.sort_records(mid["rec"], 1237, 822, 16)
    P = mid_sorted["count"]
    assert P >= len(want_vals) > 2_000_000
    extra = pu.check_lists(mid_sorted["vals"].cpu().numpy()[:P], mid_sorted["ranges"].cpu().numpy(), want_vals,
                           want_ranges, mid["rec"], 16, mid["gcam"].tiles_x)
    assert extra <= 0.02 * len(want_vals)
    assert lib.gs_get_device_error() == 0


@pytest.fixture(scope="module")
def mid_render(mid, mid_sorted):
    H, W = 822, 1237
    img = torch.zeros((3, H, W), device=DEV)
    tf = torch.zeros((H, W), device=DEV)
    nl = torch.zeros((H, W), dtype=torch.int32, device=DEV)
    lib.gs_render_fwd(mid_sorted["spl"], mid_sorted["vals"], mid_sorted["ranges"], mid["gcam"], img, tf, nl)
    torch.cuda.synchronize()
    return dict(img=img, tf=tf, nl=nl)


def test_fullsize_render_sampled_pixels(mid, mid_sorted, mid_render):
    g = np.random.default_rng(11)
    k = 20000
    px, py = g.integers(0, 1237, k), g.integers(0, 822, k)
    vals = mid_sorted["vals"].cpu().numpy()[:mid_sorted["count"]].view(np.uint32)
    ranges = mid_sorted["ranges"].cpu().numpy().view(np.uint32)
    want = oracle.render_pixels(mid["proj"], vals, ranges, mid["ocam"], px, py)
    img = mid_render["img"].cpu().numpy()[:, py, px]
    tf = mid_render["tf"].cpu().numpy()[py, px]
    nl = mid_render["nl"].cpu().numpy()[py, px]
    ok = want["margin"] > pu.PIXEL_MARGIN
    assert ok.mean() > 0.99
    assert np.array_equal(nl[ok], want["n_last"][ok])
    good, worst = pu.close(img, want["image"], 1e-4, 1.0, np.broadcast_to(ok, img.shape))
    assert good, worst
    good, worst = pu.close(tf, want["t_final"], 1e-4, 1e-3, ok)
    assert good, worst


def test_fullsize_loss(mid_render):
    """Eq. 3 over the whole 1237x822 view against a target image."""
    x = mid_render["img"].cpu().numpy().astype(np.float64)
    y = pu.f32(np.clip(x + np.random.default_rng(3).normal(0, 0.05, x.shape), 0, 1))
    Lw, dw = oracle.loss(x, y)
    H, W = 822, 1237
    ws = torch.zeros(lib.gs_loss_workspace_bytes(H, W), dtype=torch.uint8, device=DEV)
    loss = torch.zeros(1, device=DEV)
    dl = torch.zeros((3, H, W), device=DEV)
    lib.gs_loss(mid_render["img"], torch.from_numpy(y.astype(np.float32)).to(DEV), H, W, 0.2, ws, loss, dl)
    assert float(loss.item()) == pytest.approx(Lw, rel=1e-5)
    good, worst = pu.close(dl.cpu().numpy(), dw, 1e-3, np.abs(dw).mean())
    assert good, worst


def test_fullsize_backward_sampled_gaussians(mid, mid_sorted, mid_render):
    """Raster and projection backward for 60 sampled visible Gaussians: the
    oracle runs its backward over the union of their tiles only, which holds
    every pixel they touch, so their gradients are complete."""
    H, W = 822, 1237
    g = np.random.default_rng(5)
    vis = np.nonzero((mid["pr"]["radius"] > 0) & (mid["pr"]["margin"] > pu.PROJ_MARGIN))[0]
    sample = np.sort(g.choice(vis, 60, replace=False))
    tx = (W + 15) // 16
    mask = np.zeros(mid["gcam"].tiles, np.uint8)
    for i in sample:
        x0, y0, x1, y1 = mid["pr"]["rect"][i]
        for yy in range(y0, y1):
            mask[yy * tx + x0: yy * tx + x1] = 1
    dl = pu.f32(np.random.default_rng(6).normal(0, 1e-6, (3, H, W)))
    vals = mid_sorted["vals"].cpu().numpy()[:mid_sorted["count"]].view(np.uint32)
    ranges = mid_sorted["ranges"].cpu().numpy().view(np.uint32)
    # ambiguous pixels from the oracle's own forward over the masked tiles
    pix = np.nonzero(np.repeat(np.repeat(mask.reshape(-1, tx), 16, 0), 16, 1)[:H, :W])
    fwd = oracle.render_pixels(mid["proj"], vals, ranges, mid["ocam"], pix[1], pix[0])
    amb = np.zeros((H, W), np.uint8)
    amb[pix[0], pix[1]] = fwd["margin"] <= pu.PIXEL_MARGIN
    want = oracle.render_bwd(mid["proj"], vals, ranges, mid["ocam"], dl, None, amb, tile_mask=mask)
    n = mid["P"].shape[0]
    g2 = torch.zeros((n, 12), device=DEV)
    lib.gs_raster_bwd(mid_sorted["spl"], mid_sorted["vals"], mid_sorted["ranges"], mid["gcam"], mid_render["tf"],
                      mid_render["nl"], torch.from_numpy(dl.astype(np.float32)).to(DEV), None, g2)
    got = g2.cpu().numpy()[sample]
    W9 = pu.grad2d_matrix(want)[sample]
    for cols in (slice(0, 2), slice(2, 5), slice(5, 6), slice(6, 9)):
        w = W9[:, cols]
        good, worst = pu.close_bound(got[:, cols], w, 1e-3, 1e-2 * np.abs(w).max(), want["amb_abs"][sample, cols])
        assert good, (cols, worst)

    # projection backward for the same Gaussians from the oracle's raster gradients
    grads2d = dict(d_mean2d=np.zeros((n, 2)), d_conic=np.zeros((n, 3)), d_opacity=np.zeros(n), d_rgb=np.zeros((n, 3)))
    g2in = np.zeros((n, 12), np.float32)
    for key, sl in (("d_mean2d", slice(0, 2)), ("d_conic", slice(2, 5)), ("d_rgb", slice(6, 9))):
        grads2d[key][sample] = pu.f32(want[key][sample])
        g2in[sample, sl] = grads2d[key][sample]
    grads2d["d_opacity"][sample] = pu.f32(want["d_opacity"][sample])
    g2in[sample, 5] = grads2d["d_opacity"][sample]
    frozen = np.ones(n, np.uint8)
    frozen[sample] = 0
    wantG = oracle.project_bwd(mid["P"][sample], mid["ocam"], {k: v[sample] for k, v in grads2d.items()})["G"]
    Pt = torch.from_numpy(pu.pack64(mid["P"])).to(DEV)
    spl = torch.zeros((n, 12), device=DEV)
    lib.gs_project(Pt, n, 3, mid["gcam"], spl)
    G = torch.zeros((n, 64), device=DEV)
    act = torch.from_numpy(sample.astype(np.int32)).to(DEV)
    lib.gs_project_bwd(Pt, n, 3, mid["gcam"], spl, act, torch.tensor([len(sample)], dtype=torch.int32, device=DEV),
                       torch.from_numpy(g2in).to(DEV), G)
    Gs = G.cpu().numpy()[sample, :59]
    for sl in [slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11), slice(11, 14), slice(14, 59)]:
        good, worst = pu.close(Gs[:, sl], wantG[:, sl], 1e-3, 1e-2 * np.abs(wantG[:, sl]).max())
        assert good, (sl, worst)


def test_fullsize_freeze_and_adam(mid):
    """Freeze update over all 1M Gaussians (bit-exact) and Adam on sampled rows of the active list."""
    n = mid["P"].shape[0]
    g = np.random.default_rng(9)
    acc_x = (g.exponential(3e-7, n) * g.integers(0, 5, n)).astype(np.float32)
    acc_r = (g.exponential(4e-9, n) * g.integers(0, 5, n)).astype(np.float32)
    cnt = g.integers(0, 5, n).astype(np.int32)
    frozen = (g.uniform(0, 1, n) < 0.3).astype(np.uint8)
    t = [torch.from_numpy(a.copy()).to(DEV) for a in (acc_x, acc_r, cnt, frozen)]
    act = torch.zeros(n, dtype=torch.int32, device=DEV)
    na = torch.zeros(1, dtype=torch.int32, device=DEV)
    ws = torch.zeros(lib.gs_freeze_workspace_bytes(n), dtype=torch.uint8, device=DEV)
    lib.gs_freeze_update(n, *t, 3e-7, 4e-9, 0, act, na, ws)
    want_act = oracle.freeze_update(acc_x, acc_r, cnt, frozen, np.float32(3e-7), np.float32(4e-9), 0)
    k = int(na.item())
    assert k == len(want_act) and np.array_equal(act.cpu().numpy()[:k], want_act)
    assert np.array_equal(t[3].cpu().numpy(), frozen)

    rows = np.sort(g.choice(want_act, 5000, replace=False))
    P = pu.f32(mid["P"][rows])
    Gr = pu.f32(g.normal(0, 1e-4, P.shape))
    Pt = torch.from_numpy(pu.pack64(mid["P"])).to(DEV)
    Gt = torch.zeros_like(Pt)
    Gt[torch.from_numpy(rows).to(DEV), :59] = torch.from_numpy(Gr.astype(np.float32)).to(DEV)
    Mt, Vt = torch.zeros_like(Pt), torch.zeros_like(Pt)
    lrs = [float(np.float32(x)) for x in pipeline.default_lrs(4.4)]
    b1, b2, eps = float(np.float32(0.9)), float(np.float32(0.999)), float(np.float32(1e-15))
    lib.gs_adam_masked(Pt, Gt, Mt, Vt, n, torch.from_numpy(rows.astype(np.int32)).to(DEV),
                       torch.tensor([len(rows)], dtype=torch.int32, device=DEV), lrs, b1, b2, eps, 1)
    Po, Mo, Vo = P.copy(), np.zeros_like(P), np.zeros_like(P)
    oracle.adam(Po, Gr, Mo, Vo, None, np.array(lrs), 1, b1=b1, b2=b2, eps=eps)
    got = Pt.cpu().numpy()
    assert np.allclose(got[rows, :59], Po, rtol=0, atol=1e-6 * (1 + np.abs(Po).max()))
    others = np.setdiff1d(np.arange(n), rows)[:100000]
    assert np.array_equal(got[others, :59], mid["P"][others].astype(np.float32))


def test_fullsize_psnr(mid_render):
    x = mid_render["img"]
    y = (x + 0.03).clamp(0, 1)
    ws = torch.zeros(lib.gs_psnr_workspace_bytes(1, 822, 1237), dtype=torch.uint8, device=DEV)
    out = torch.zeros(1, device=DEV)
    lib.gs_psnr(x, y, 1, 822, 1237, ws, out)
    want = oracle.psnr(x.cpu().numpy()[None].astype(np.float64), y.cpu().numpy()[None].astype(np.float64))[0]
    assert float(out.item()) == pytest.approx(want, abs=1e-3)
