"""The torch.autograd wrappers: the hand-written backward behind
RasterizeGaussians / SsimL1Loss gives the oracle's gradient."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2504_06716_gb300 import autograd, lib, synth  # noqa: E402

import parity_util as pu  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06716_gb300 import build

    build.build()
    oracle.build()
    lib.load()


def _nudge(P, ocam):
    for _ in range(20):
        bad = oracle.project(P, ocam)["margin"] <= pu.PROJ_MARGIN
        if not bad.any():
            return P
        P = P.copy()
        P[bad, 3:6] += 3e-3
        P = pu.f32(P)
    raise AssertionError("nudge failed")


def test_autograd_gradient_matches_oracle_with_frozen_rows():
    s = synth.tiny_scene(seed=2)
    ocam, gcam = pu.cameras(s.cameras[1])
    P = _nudge(pu.f32(s.init), ocam)
    gt = pu.f32(oracle.forward(pu.f32(s.gt), ocam)["image"])
    frozen = (np.random.default_rng(1).uniform(size=P.shape[0]) < 0.25).astype(np.uint8)
    Pt = torch.from_numpy(pu.pack64(P)).cuda().requires_grad_(True)
    image = autograd.rasterize(Pt, gcam, frozen=torch.from_numpy(frozen).cuda())
    loss = autograd.ssim_l1_loss(image, torch.from_numpy(gt.astype(np.float32)).cuda())
    loss.backward()
    G = Pt.grad.cpu().numpy()[:, :59]
    want = oracle.loss_and_grad(P, ocam, gt, frozen=frozen)
    assert float(loss.item()) == pytest.approx(want["loss"], rel=1e-4)
    amb = (want["fwd"]["margin"] <= pu.E2E_PIXEL_MARGIN).astype(np.uint8)
    rb = oracle.render_bwd(want["fwd"]["proj"], want["fwd"]["vals"], want["fwd"]["ranges"], ocam, want["dl_dimage"],
                           frozen, amb)
    l1 = pu.l1_sign_bound(want["fwd"]["proj"], want["fwd"]["vals"], want["fwd"]["ranges"], ocam, want["fwd"]["image"],
                          gt, frozen)
    bound = pu.param_bound(P, ocam, rb["amb_abs"] + l1, frozen)
    assert np.all(G[frozen == 1] == 0)
    act = frozen == 0
    for sl in [slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11), slice(11, 14), slice(14, 59)]:
        w = want["G"][act, sl]
        good, worst = pu.close_bound(G[act, sl], w, 1e-3, 1e-2 * np.abs(w).max(), bound[act, sl])
        assert good, (sl, worst)
    assert np.all(Pt.grad.cpu().numpy()[:, 59:] == 0)
