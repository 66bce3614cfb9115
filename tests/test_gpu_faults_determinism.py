"""Host-made faults and repeat-run determinism of the CUDA path.

Faults are made on the host (non-finite values in an input image); the device
error word must record them and its read must clear it. No test here makes a
kernel fault, trap or wait.

Determinism: projection, sort, compositing and the loss use no floating-point
atomics, so two runs on the same inputs give the same bytes. The rasteriser
backward adds per-tile partial sums into the per-Gaussian gradient with
atomics, so repeat runs may differ by the order of those additions only.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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
    lib.load()
    lib.gs_get_device_error()  # start from a clear error word


def _loss(x, y, lam=0.2):
    H, W = x.shape[1], x.shape[2]
    xt = torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(DEV)
    yt = torch.from_numpy(np.ascontiguousarray(y, np.float32)).to(DEV)
    ws = torch.zeros(lib.gs_loss_workspace_bytes(H, W), dtype=torch.uint8, device=DEV)
    loss = torch.zeros(1, device=DEV)
    dl = torch.zeros_like(xt)
    lib.gs_loss(xt, yt, H, W, lam, ws, loss, dl)
    torch.cuda.synchronize()
    return float(loss.item()), dl.cpu().numpy()


@pytest.mark.parametrize("where", ["target", "image"])
@pytest.mark.parametrize("value", [np.nan, np.inf])
def test_nonfinite_input_raises_the_flag_and_the_read_clears_it(where, value):
    g = np.random.default_rng(11)
    x = g.uniform(0, 1, (3, 45, 70)).astype(np.float32)
    y = np.clip(x + g.normal(0, 0.1, x.shape), 0, 1).astype(np.float32)
    (y if where == "target" else x)[1, 20, 33] = value
    L, _ = _loss(x, y)
    assert not np.isfinite(L)
    flags = lib.gs_get_device_error()
    assert flags & lib.GS_FLAG_NONFINITE
    assert not flags & (lib.GS_FLAG_CAPACITY | lib.GS_FLAG_BADJOB)
    assert lib.gs_get_device_error() == 0  # cleared by the read
    # the context is still usable: a clean call afterwards is finite and raises nothing
    y[np.isfinite(y) == 0] = 0.5
    x[np.isfinite(x) == 0] = 0.5
    L2, dl2 = _loss(x, y)
    assert np.isfinite(L2) and np.isfinite(dl2).all()
    assert lib.gs_get_device_error() == 0


def _forward(P, gcam, capacity):
    n = P.shape[0]
    Pt = torch.from_numpy(pu.pack64(P)).to(DEV)
    spl = torch.zeros((n, 12), dtype=torch.float32, device=DEV)
    lib.gs_project(Pt, n, 3, gcam, spl)
    ws = torch.zeros(lib.gs_sort_workspace_bytes(n, capacity, gcam), dtype=torch.uint8, device=DEV)
    vals = torch.full((capacity,), -1, dtype=torch.int32, device=DEV)
    ranges = torch.full((gcam.tiles, 2), -1, dtype=torch.int32, device=DEV)
    count = torch.zeros(1, dtype=torch.int64, device=DEV)
    lib.gs_sort(spl, n, gcam, ws, capacity, vals, ranges, count)
    H, W = gcam.height, gcam.width
    img = torch.zeros((3, H, W), device=DEV)
    tf = torch.zeros((H, W), device=DEV)
    nl = torch.zeros((H, W), dtype=torch.int32, device=DEV)
    lib.gs_render_fwd(spl, vals, ranges, gcam, img, tf, nl)
    torch.cuda.synchronize()
    return dict(spl=spl, vals=vals, ranges=ranges, count=count, img=img, tf=tf, nl=nl)


def _backward(out, gcam, dl, frozen):
    n = out["spl"].shape[0]
    g2 = torch.zeros((n, 12), device=DEV)
    lib.gs_raster_bwd(out["spl"], out["vals"], out["ranges"], gcam, out["tf"], out["nl"], dl, frozen, g2)
    torch.cuda.synchronize()
    return g2.cpu().numpy()


@pytest.mark.parametrize("tile", [8, 16])
def test_repeat_runs_forward_bit_identical_backward_within_rounding(tile):
    s = synth.surface_scene(6000, 10, 8, 320, 214, seed=5)
    P = pu.f32(s.init)
    _, gcam = pu.cameras(s.cameras[3], tile=tile)
    capacity = 200_000
    a = _forward(P, gcam, capacity)
    b = _forward(P, gcam, capacity)
    Pn = int(a["count"].item())
    assert 0 < Pn <= capacity and int(b["count"].item()) == Pn
    for k in ("spl", "ranges", "img", "tf", "nl"):
        assert torch.equal(a[k], b[k]), k
    assert torch.equal(a["vals"][:Pn], b["vals"][:Pn])
    gt = torch.clamp(a["img"] + 0.05 * torch.sin(torch.arange(a["img"].numel(), device=DEV).view_as(a["img"])),
                     0, 1)
    La, dla = _loss(a["img"].cpu().numpy(), gt.cpu().numpy())
    Lb, dlb = _loss(b["img"].cpu().numpy(), gt.cpu().numpy())
    assert La == Lb and np.array_equal(dla, dlb)
    dl = torch.from_numpy(dla).to(DEV)
    frozen = torch.from_numpy((np.random.default_rng(4).uniform(0, 1, P.shape[0]) < 0.3).astype(np.uint8)).to(DEV)
    ga, gb = _backward(a, gcam, dl, frozen), _backward(b, gcam, dl, frozen)
    assert np.array_equal(ga == 0, gb == 0)  # the same Gaussians receive gradient
    for cols in (slice(0, 2), slice(2, 5), slice(5, 6), slice(6, 9)):
        scale = np.abs(ga[:, cols]).max()
        assert np.abs(ga[:, cols] - gb[:, cols]).max() <= 1e-5 * scale, cols
    assert lib.gs_get_device_error() == 0
