"""Volume masks (Sec. 3.3, "Pruning with Volume Masking") through the C ABI
against the oracle: masked-off Gaussians culled in the projection (the rest
bit for bit as without masks), the mask logit's straight-through gradient,
the seventh Adam group, pruning of masked-off Gaussians, a short training
run with masks."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import densify as D  # noqa: E402
from paper_2504_06716_gb300 import lib, synth  # noqa: E402

import parity_util as pu  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"
LOGIT_MIN = float(np.float32(math.log(0.01 / 0.99)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06716_gb300 import build

    build.build()
    oracle.build()
    lib.load()


def _case(n=6000, seed=5):
    s = synth.surface_scene(n, 10, 8, 320, 214, seed=seed)
    P = pu.f32(s.init)
    g = np.random.default_rng(seed)
    mask = g.uniform(-8.0, 4.0, n).astype(np.float32)
    mask[:4] = [LOGIT_MIN, np.nextafter(np.float32(LOGIT_MIN), np.float32(1)), -20.0, 20.0]
    return P, mask.astype(np.float64), s.cameras


def _packed(P, mask):
    R = pu.pack64(P)
    R[:, 59] = mask.astype(np.float32)
    return torch.from_numpy(R).to(DEV)


def test_projection_culls_masked_off_gaussians():
    P, mask, cams = _case()
    n = P.shape[0]
    ocam, gcam = pu.cameras(cams[1])
    Pt = _packed(P, mask)
    a, b = torch.zeros((n, 12), device=DEV), torch.zeros((n, 12), device=DEV)
    lib.gs_project_ex(Pt, n, 3, lib.GS_VOLUME_MASK, gcam, a)
    lib.gs_project_ex(Pt, n, 3, 0, gcam, b)
    a, b = a.cpu().numpy(), b.cpu().numpy()
    off = ~(mask.astype(np.float32) > np.float32(LOGIT_MIN))
    assert off[0] and not off[1] and off.sum() > 1000
    assert np.all(a[off] == 0) and np.array_equal(a[~off], b[~off])
    want = oracle.project(P, ocam, mask=mask)
    assert np.array_equal(want["radius"][off], np.zeros(off.sum(), np.int32))


def test_mask_gradient_matches_oracle():
    P, mask, cams = _case(seed=6)
    n = P.shape[0]
    ocam, gcam = pu.cameras(cams[2])
    g = np.random.default_rng(7)
    g2 = pu.f32(g.normal(0, 1e-3, (n, 12)))
    g2[:, 9:] = 0
    grads2d = dict(d_mean2d=g2[:, 0:2], d_conic=g2[:, 2:5], d_opacity=g2[:, 5], d_rgb=g2[:, 6:9])
    frozen = (g.uniform(size=n) < 0.2).astype(np.uint8)
    lam = float(np.float32(5e-4 / n))
    want = oracle.project_bwd(P, ocam, grads2d, frozen=frozen, mask=mask, mask_loss=lam)
    Pt = _packed(P, mask)
    spl = torch.zeros((n, 12), device=DEV)
    lib.gs_project_ex(Pt, n, 3, lib.GS_VOLUME_MASK, gcam, spl)
    G = torch.full((n, 64), 9.0, device=DEV)
    act = torch.from_numpy(np.nonzero(frozen == 0)[0].astype(np.int32)).to(DEV)
    na = torch.tensor([act.numel()], dtype=torch.int32, device=DEV)
    lib.gs_project_bwd_ex(Pt, n, 3, lib.GS_VOLUME_MASK, gcam, spl, act, na,
                          torch.from_numpy(g2.astype(np.float32)).to(DEV), G, False, [], lam)
    G = G.cpu().numpy()
    fr = frozen == 1
    assert np.all(G[fr] == 9.0)  # frozen rows untouched
    proj = oracle.project(P, ocam, mask=mask)
    safe = proj["margin"] > pu.PROJ_MARGIN
    a = ~fr & safe
    w = want["G_mask"][a]
    good, worst = pu.close(G[a, 59], w, 1e-3, 1e-2 * np.abs(w).max())
    assert good, worst
    vis = a & (proj["radius"] > 0)
    for sl in (slice(0, 3), slice(3, 6), slice(10, 11)):
        ww = want["G"][vis, sl]
        good, worst = pu.close(G[vis, sl], ww, 1e-3, 1e-2 * np.abs(ww).max())
        assert good, (sl, worst)


def test_seventh_adam_group_moves_the_mask_logit():
    n = 1000
    g = np.random.default_rng(3)
    P = torch.from_numpy(g.normal(0, 1, (n, 64)).astype(np.float32)).to(DEV)
    G = torch.zeros((n, 64), device=DEV)
    G[:, 59] = torch.from_numpy(g.normal(0, 1, n).astype(np.float32)).to(DEV)
    m, v = torch.zeros_like(P), torch.zeros_like(P)
    act = torch.arange(n, dtype=torch.int32, device=DEV)
    na = torch.tensor([n], dtype=torch.int32, device=DEV)
    P0 = P.clone()
    lr = [1e-3, 5e-3, 1e-3, 0.025, 2.5e-3, 1.25e-4, 0.01]
    lib.gs_adam_masked_groups(P, G, m, v, n, act, na, lr, 0.9, 0.999, 1e-15, 1)
    d = (P - P0).cpu().numpy()
    # first step: m_hat / sqrt(v_hat) = sign(g): the logit moves by the rate
    gm = G[:, 59].cpu().numpy()
    assert np.allclose(d[:, 59], -0.01 * np.sign(gm), rtol=1e-5, atol=0)
    assert not d[:, :59].any() and not d[:, 60:].any()
    P1 = P.clone()
    lib.gs_adam_masked_groups(P, G, m, v, n, act, na, lr[:6], 0.9, 0.999, 1e-15, 2)  # six groups: 59 stays
    assert torch.equal(P[:, 59], P1[:, 59])


def test_prune_masked_matches_oracle():
    P, mask, _ = _case(n=20011, seed=8)
    n = P.shape[0]
    P64 = np.concatenate([P, mask[:, None].astype(np.float32).astype(np.float64)], axis=1)
    prm = D.DensifyParams(eps_xyz=float("inf"), eps_rgb=float("inf"), use_rgb=False, log_clone_max=0.0,
                          logit_min_opacity=float("-inf"), prune_big=False, max_screen_radius=2**31 - 1,
                          log_max_world=float("inf"), log_split_div=0.0, mask_prune=True, mask_logit_min=LOGIT_MIN)
    want = D.densify(P64, np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n, int), prm, np.zeros((0, 2, 3)))
    from paper_2504_06716_gb300 import pipeline
    mdl = pipeline.Model(P, device=DEV)
    mdl.P[:n, 59] = torch.from_numpy(mask.astype(np.float32)).to(DEV)
    res = mdl.prune_masked(LOGIT_MIN, np.random.default_rng(0))
    assert res["n"] == len(want["src"]) and res["kept"] == len(want["src"])
    assert np.array_equal(mdl.P[: res["n"], :60].cpu().numpy().astype(np.float64), want["P"])
    assert int(mdl.n_active.item()) == res["n"]


def test_training_with_volume_masks():
    from paper_2504_06716_gb300.schedule import GStaConfig
    from paper_2504_06716_gb300.train import Trainer

    cfg = GStaConfig.tiny()
    cfg.volume_mask, cfg.mask_from, cfg.mask_until, cfg.mask_prune_every, cfg.mask_lambda = True, 10, 100, 30, 0.5
    cfg.mask_lr = 0.2  # fast enough for a tiny run to switch masks off
    tr = Trainer(synth.tiny_scene(), cfg, tile=16)
    n0 = tr.model.n
    while tr.k < 110:
        tr.iteration()
    assert any(e[1] == "mask_prune" for e in tr.events)
    assert tr.model.n < n0
    assert lib.gs_get_device_error() == 0
    assert np.isfinite(tr.heldout_psnr())
