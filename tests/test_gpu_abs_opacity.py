"""Absolute-value opacity of the finetuning stage (Sec. 4.1) through the C
ABI against the oracle: projection with opacity = |x|, the gradient through
|x|, and the switch gs_opacity_to_abs (every splat record bit for bit the
same before and after); a short training run that enters finetuning."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import densify as D  # noqa: E402
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


def _params(n=6000, seed=5):
    s = synth.surface_scene(n, 10, 8, 320, 214, seed=seed)
    P = pu.f32(s.init)
    g = np.random.default_rng(seed)
    P[:, 10] = pu.f32(g.uniform(0.02, 1.6, n) * g.choice([-1.0, 1.0], n))  # |x| also above 1
    return P, s.cameras


def _project(P, gcam, act):
    n = P.shape[0]
    Pt = torch.from_numpy(pu.pack64(P)).to(DEV)
    spl = torch.zeros((n, 12), device=DEV)
    lib.gs_project_ex(Pt, n, 3, act, gcam, spl)
    return Pt, spl


def test_project_abs_matches_oracle():
    P, cams = _params()
    ocam, gcam = pu.cameras(cams[1])
    want = oracle.project(P, ocam, opacity_act=1)
    _, spl = _project(P, gcam, lib.GS_OPACITY_ABS)
    got = spl.cpu().numpy()
    vis = (want["margin"] > pu.PROJ_MARGIN) & (want["radius"] > 0)
    assert vis.sum() > 500
    assert np.array_equal(got[vis, 5], np.abs(P[vis, 10]).astype(np.float32))  # exact
    assert (got[vis, 5] > 1).any()
    _, spl_s = _project(P, gcam, lib.GS_OPACITY_SIGMOID)  # only the opacity column differs
    a, b = got.copy(), spl_s.cpu().numpy()
    a[:, 5] = b[:, 5] = 0
    assert np.array_equal(a, b)


def test_project_backward_abs_matches_oracle():
    P, cams = _params(seed=6)
    n = P.shape[0]
    ocam, gcam = pu.cameras(cams[2])
    g = np.random.default_rng(7)
    g2 = pu.f32(g.normal(0, 1e-3, (n, 12)))
    g2[:, 9:] = 0
    grads2d = dict(d_mean2d=g2[:, 0:2], d_conic=g2[:, 2:5], d_opacity=g2[:, 5], d_rgb=g2[:, 6:9])
    want = oracle.project_bwd(P, ocam, grads2d, opacity_act=1)
    Pt, spl = _project(P, gcam, lib.GS_OPACITY_ABS)
    G = torch.zeros((n, 64), device=DEV)
    act = torch.arange(n, dtype=torch.int32, device=DEV)
    na = torch.tensor([n], dtype=torch.int32, device=DEV)
    lib.gs_project_bwd_ex(Pt, n, 3, lib.GS_OPACITY_ABS, gcam, spl, act, na,
                          torch.from_numpy(g2.astype(np.float32)).to(DEV), G, False, [])
    G = G.cpu().numpy()
    proj = oracle.project(P, ocam, opacity_act=1)
    vis = (proj["margin"] > pu.PROJ_MARGIN) & (spl.cpu().numpy()[:, 10].view(np.int32) > 0)
    # the opacity column is sign(x) dL/do exactly (a float32 product with +-1)
    assert np.array_equal(G[vis, 10], (np.sign(P[vis, 10]) * g2[vis, 5]).astype(np.float32))
    assert np.array_equal(G[vis, 10].astype(np.float64), want["G"][vis, 10])
    for sl in (slice(0, 3), slice(3, 6), slice(6, 10), slice(11, 59)):
        w = want["G"][vis, sl]
        good, worst = pu.close(G[vis, sl], w, 1e-3, 1e-2 * np.abs(w).max())
        assert good, (sl, worst)


@pytest.mark.parametrize("moments", [0, 1])
def test_switch_keeps_every_splat_record(moments):
    P, cams = _params(seed=8)
    P[:, 10] = pu.f32(np.random.default_rng(9).normal(0, 3, P.shape[0]))  # logits
    n = P.shape[0]
    _, gcam = pu.cameras(cams[0])
    Pt, before = _project(P, gcam, lib.GS_OPACITY_SIGMOID)
    g = np.random.default_rng(10)
    m = torch.from_numpy(g.normal(0, 1, (n, 64)).astype(np.float32)).to(DEV)
    v = torch.from_numpy(g.uniform(0, 1, (n, 64)).astype(np.float32)).to(DEV)
    m0, v0 = m.clone(), v.clone()
    slope = torch.zeros(1, device=DEV)
    lib.gs_opacity_to_abs(n, Pt, m, v, moments, slope)
    after = torch.zeros_like(before)
    lib.gs_project_ex(Pt, n, 3, lib.GS_OPACITY_ABS, gcam, after)
    assert torch.equal(after, before)
    keep = torch.ones(64, dtype=torch.bool, device=DEV)
    keep[10] = False
    assert torch.equal(m[:, keep], m0[:, keep]) and torch.equal(v[:, keep], v0[:, keep])
    M = np.zeros((n, 59))
    V = np.zeros((n, 59))
    M[:, 10] = m0[:n, 10].cpu().numpy()
    V[:, 10] = v0[:n, 10].cpu().numpy()
    Q = P.copy()
    D.opacity_to_abs(Q, M, V, rescale=bool(moments))
    got = Pt[:n, 10].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - Q[:, 10]) <= 4 * np.spacing(np.abs(Q[:, 10]).astype(np.float32)))
    want_slope = float(np.sum(Q[:, 10] * (1 - Q[:, 10])))
    assert abs(float(slope.item()) - want_slope) <= 1e-4 * want_slope
    if moments:
        # s = o (1 - o) from the float32 o: its relative error is about
        # eps (1/o + 1/(1 - o)) (cancellation in 1 - o), twice that for v
        o = Q[:, 10]
        rel = 8 * 2.0 ** -24 * (1 / o + 1 / (1 - o)) + 1e-6
        for t, w, k in ((m, M, 1), (v, V, 2)):
            g = t[:n, 10].cpu().numpy().astype(np.float64)
            assert np.all(np.abs(g - w[:, 10]) <= k * rel * np.abs(w[:, 10]) + 1e-30)
    else:
        assert not m[:, 10].any() and not v[:, 10].any()


def test_invalid_activation_is_rejected():
    P, cams = _params(n=100)
    _, gcam = pu.cameras(cams[0])
    Pt = torch.from_numpy(pu.pack64(P)).to(DEV)
    spl = torch.zeros((100, 12), device=DEV)
    with pytest.raises(lib.GsError):
        lib.gs_project_ex(Pt, 100, 3, 4, gcam, spl)  # no such flag


def test_training_enters_finetune_with_abs_opacity():
    """The tiny schedule to its end: the finetuning stage switches the
    activation, the image is unchanged by the switch and training goes on."""
    from paper_2504_06716_gb300.schedule import GStaConfig
    from paper_2504_06716_gb300.train import Trainer

    scene = synth.tiny_scene()
    tr = Trainer(scene, GStaConfig.tiny(), tile=16)
    while tr.ctrl.finetune_left is None:
        tr.iteration()
    assert tr.model.opacity_act == lib.GS_OPACITY_ABS
    assert any(e[1] == "abs_opacity" for e in tr.events)
    while not tr.finished():
        tr.iteration()
    assert lib.gs_get_device_error() == 0
    assert np.isfinite(tr.heldout_psnr())
