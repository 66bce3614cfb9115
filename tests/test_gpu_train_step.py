"""gs_train_step (the whole inner step enqueued from native code) against the
same entry points called one by one from Python: identical forward outputs
and lists, and the same update up to the order of the rasteriser's atomic
additions; argument validation."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2504_06716_gb300 import lib, pipeline, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06716_gb300 import build

    build.build()
    lib.load()


def _model(scene, densify, frozen_every=0):
    m = pipeline.Model(scene.init, device=DEV, capacity=int(scene.init.shape[0] * 1.5))
    if densify:
        m.enable_densify()
    if frozen_every:
        m.frozen[: m.n : frozen_every] = 1
        m.freeze_update(0.0, 0.0, 3)
    return m


@pytest.mark.parametrize("densify,frozen_every", [(False, 0), (True, 3)])
def test_native_step_matches_the_piecewise_step(densify, frozen_every):
    scene = synth.surface_scene(20000, 30000, 6, 320, 214, seed=2)
    cams = [lib.camera(c, tile=16) for c in scene.cameras]
    gt = torch.rand((3, 214, 320), device=DEV)
    lrs = pipeline.default_lrs(4.4)
    a, b = _model(scene, densify, frozen_every), _model(scene, densify, frozen_every)
    cap = a.measure_capacity(cams)
    va, vb = a.make_view(cams[0], cap), b.make_view(cams[0], cap)
    for k in range(4):
        # same state on both sides before each step (the rasteriser backward's
        # atomic additions make the two updates differ in the last bits)
        for x, y in ((a.P, b.P), (a.m, b.m), (a.v, b.v), (a.acc_xyz, b.acc_xyz), (a.acc_rgb, b.acc_rgb),
                     (a.cnt, b.cnt)):
            y.copy_(x)
        if densify:
            for key in ("acc_xyz", "acc_rgb", "cnt", "max_radius"):
                b.den[key].copy_(a.den[key])
        cam = cams[k % len(cams)]
        a.retarget(va, cam)
        b.retarget(vb, cam)
        a.train_step(va, gt, lrs)  # native
        b.rasterize(vb)
        b.loss(vb, gt)
        b.backward(vb)
        b.adam(lrs)
        torch.cuda.synchronize()
        assert torch.equal(va.image, vb.image) and torch.equal(va.n_last, vb.n_last)
        assert torch.equal(va.count, vb.count) and torch.equal(va.ranges, vb.ranges)
        assert torch.equal(va.vals[: int(va.count)], vb.vals[: int(vb.count)])
        assert torch.equal(va.loss, vb.loss)
        assert torch.equal(a.cnt, b.cnt)
        for x, y in ((a.P, b.P), (a.m, b.m), (a.v, b.v), (a.acc_xyz, b.acc_xyz)):
            scale = y.abs().max().item() + 1e-30
            assert (x - y).abs().max().item() <= 1e-5 * scale
        if densify:
            assert torch.equal(a.den["cnt"], b.den["cnt"])
        assert a.step_count == b.step_count == k + 1
    assert lib.gs_get_device_error() == 0


def test_native_step_rejects_bad_arguments():
    scene = synth.tiny_scene()
    m = _model(scene, False)
    cam = lib.camera(scene.cameras[0], tile=16)
    v = m.make_view(cam, m.measure_capacity([cam]))
    gt = torch.zeros((3, cam.height, cam.width), device=DEV)
    st = m._step_struct(v)
    with pytest.raises(lib.GsError):
        lib.gs_train_step(st, cam, gt, pipeline.default_lrs(4.4), 0)  # Adam step must be >= 1
    st.n_stats = 3
    with pytest.raises(lib.GsError):
        lib.gs_train_step(st, cam, gt, pipeline.default_lrs(4.4), 1)


def test_target_feeder_delivers_each_step_its_image():
    """Double-buffered uploads: every take() returns the image prefetched for
    that step, with the next upload in flight during the step."""
    g = np.random.default_rng(4)
    imgs = [torch.from_numpy(g.uniform(0, 1, (3, 96, 128)).astype(np.float32)) for _ in range(6)]
    host = [x.pin_memory() for x in imgs]
    feeder = pipeline.TargetFeeder((3, 96, 128))
    sink = torch.zeros((3, 96, 128), device=DEV)
    feeder.prefetch(host[0])
    for i in range(6):
        t = feeder.take()
        sink.copy_(t)  # the step's use of its target
        sink.mul_(1.0)
        feeder.release()
        if i + 1 < 6:
            feeder.prefetch(host[i + 1])
        torch.cuda.current_stream().synchronize()
        assert torch.equal(sink.cpu(), imgs[i])
