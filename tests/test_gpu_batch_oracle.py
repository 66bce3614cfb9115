"""The batched step of several uneven scenes (batch.py: per-(scene, view)
projection and sort, one persistent compositing launch and one persistent
backward launch over every job, per-scene projection backward summed over
the scene's views, device-step Adam, the whole step captured in a CUDA graph
and replayed) against the FP64 oracle of that step (oracle/batch_step.py).

Three scenes of 700, 1,600 and 3,200 Gaussians, three 76x76 views of each per
step (ragged 8- and 16-pixel tiles), the freeze schedule shortened so that
the compared step opens with a freeze update on a map the method produced.
Before the compared replay, the parameters are moved off the projection's
integer decision boundaries (as the single-step end-to-end test does) and
written back, so that both sides start from the same float32 state. Then:

* freeze map, active list and count equal the oracle's bit for bit (same
  float32 statistics and thresholds);
* each view's loss equals the oracle's within 1e-4 relative;
* the scene's gradient (the sum over its views) equals the oracle's within
  1e-3 relative (floor 1% of the largest magnitude), widened only by what
  the float32 decisions within 2e-4 of a threshold, and the L1 signs of
  Eq. 3 where image and target agree within 1e-5, may change, for every
  Gaussian farther than 0.3 from the near plane in all views (nearer, the
  float32 Jacobian terms in 1/z^2 carry per-cent errors; at most 1% of the
  Gaussians);
* visibility counts are exact and the accumulated norms within 1e-3;
* Adam from the same gradient, moments and the scene's own step counter
  equals the oracle's (tolerances of the single-step Adam test); frozen rows
  keep their parameters and moments bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import batch_step as OB  # noqa: E402
from oracle import controller as C  # noqa: E402
from paper_2504_06716_gb300 import batch, lib  # noqa: E402
from paper_2504_06716_gb300.schedule import GStaConfig  # noqa: E402

import parity_util as pu  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"

SIZES = (700, 1600, 3200)
RES = 76
SCHED = dict(total_iter=200, warmup=4, window_end=150, every=4, reset_every=80, wait=2, psnr_every=1000,
             finetune_iters=20)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06716_gb300 import build

    build.build()
    oracle.build()
    lib.load()


def _nudge(P, ocams, tries=30):
    """Move Gaussians whose radius or tile rectangle sits within PROJ_MARGIN of
    a boundary in any of the views slightly off it."""
    P = P.copy()
    for _ in range(tries):
        bad = np.zeros(P.shape[0], bool)
        for oc in ocams:
            bad |= oracle.project(P, oc)["margin"] <= pu.PROJ_MARGIN
        if not bad.any():
            return pu.f32(P)
        P[bad, 3:6] += 3e-3
        P[bad, 0] += 1e-3
        P = pu.f32(P)
    raise AssertionError("could not move every Gaussian off a decision boundary")


def _state(s):
    m = s.model
    n = m.n
    f = lambda t: t.detach().cpu().numpy().copy()  # noqa: E731
    return dict(P=f(m.P)[:n, :59], M=f(m.m)[:n, :59], V=f(m.v)[:n, :59], G=f(m.G)[:n, :59], frozen=f(m.frozen)[:n],
                act=f(m.act)[: int(m.n_active.item())], acc_x=f(m.acc_xyz)[:n], acc_r=f(m.acc_rgb)[:n],
                cnt=f(m.cnt)[:n], step=int(s.step_dev.item()), lr=f(s.lr_dev))


@pytest.mark.parametrize("tile", [8, 16])
def test_graph_replayed_batch_step_matches_oracle(tile):
    cfg = GStaConfig(densify=False, **SCHED)
    scenes = batch.make_scenes(SIZES, RES, n_views=10, seed=60)
    bt = batch.BatchTrainer(scenes, cfg, tile=tile, views_per_step=3, calibrate=True)
    k_cmp = 8  # an update (every 4 from 4); its view group was captured at k = 2 and replayed at 5
    while bt.k < k_cmp:
        bt.step("graph")
    torch.cuda.synchronize()
    assert lib.gs_get_device_error() == 0
    group = bt.group_of(k_cmp)
    assert group in bt.graphs  # the compared step is a replay
    ocfg = C.ScheduleConfig(**SCHED)
    snaps, oracle_scenes = [], []
    for s in bt.scenes:
        views = s.groups[group]
        ocams = [pu.cameras(s.scene.cameras[v], tile=tile)[0] for v in views]
        P = _nudge(s.model.P.cpu().numpy()[: s.model.n, :59].astype(np.float64), ocams)
        s.model.P[: s.model.n, :59] = torch.from_numpy(P.astype(np.float32)).to(DEV)
        st = _state(s)
        snaps.append(st)
        action = C.freeze_action(k_cmp, ocfg, s.ctrl.last_reset, s.ctrl.stop_iter)
        assert action == "update"
        ex, er = s.thresholds(k_cmp)  # the host values the step uses (schedule: test_host_controller.py)
        assert ex == pytest.approx(C.threshold(s.eps0[0], k_cmp, ocfg.total_iter), rel=1e-12)
        assert er == pytest.approx(C.threshold(s.eps0[1], k_cmp, ocfg.total_iter), rel=1e-12)
        oracle_scenes.append(dict(P=P.copy(), M=st["M"].astype(np.float64), V=st["V"].astype(np.float64),
                                  frozen=st["frozen"].copy(), acc_x=st["acc_x"].copy(), acc_r=st["acc_r"].copy(),
                                  cnt=st["cnt"].copy(), step=st["step"],
                                  lr=np.concatenate([[np.float32(s.ctrl.lr_xyz_at(k_cmp))], st["lr"][1:]]).astype(
                                      np.float64),
                                  cams=ocams, gts=[pu.f32(s.targets[v].cpu().numpy()) for v in views], action=0,
                                  eps_xyz=np.float32(ex), eps_rgb=np.float32(er)))
    assert sum(int((st["frozen"] == 1).sum()) for st in snaps) > 0  # the first update froze something
    bt.step("graph")
    torch.cuda.synchronize()
    assert lib.gs_get_device_error() == 0
    b1, b2, eps = float(np.float32(0.9)), float(np.float32(0.999)), float(np.float32(1e-15))
    want = OB.batch_step(oracle_scenes, k_cmp, b1=b1, b2=b2, eps=eps)
    for s, st0, o, w in zip(bt.scenes, snaps, oracle_scenes, want):
        got = _state(s)
        # freeze action: bit for bit
        assert np.array_equal(got["frozen"], o["frozen"])
        assert np.array_equal(got["act"], w["act"])
        fr = o["frozen"] == 1
        assert fr.any() and (~fr).any()
        # each view's loss
        for slot, wl in zip(s.slots, w["losses"]):
            assert float(slot.view.loss.item()) == pytest.approx(wl, rel=1e-4)
        # the scene's gradient: sum over its views
        n = o["P"].shape[0]
        bound = np.zeros((n, 59))
        amb_rows = np.zeros(n, bool)
        vis = np.zeros(n, bool)
        near = np.zeros(n, bool)
        for oc, o_gt, r in zip(o["cams"], o["gts"], w["views"]):
            f = r["fwd"]
            amb = f["margin"] <= pu.E2E_PIXEL_MARGIN
            assert amb.mean() < 0.05
            rb = oracle.render_bwd(f["proj"], f["vals"], f["ranges"], oc, r["dl_dimage"], o["frozen"],
                                   amb.astype(np.uint8))
            l1 = pu.l1_sign_bound(f["proj"], f["vals"], f["ranges"], oc, f["image"], o_gt, o["frozen"])
            bound += pu.param_bound(st0["P"].astype(np.float64), oc, rb["amb_abs"] + l1, o["frozen"])
            amb_rows |= rb["amb_abs"].any(axis=1) | l1.any(axis=1)
            vis |= f["proj"]["radius"] > 0
            # within 0.3 of the near plane the Jacobian's 1/z^2 terms leave float32
            # gradients with a few per cent of error: such Gaussians are left out
            near |= (f["proj"]["radius"] > 0) & (f["proj"]["depth"] < 0.5)
        assert near.sum() <= 0.01 * n
        act = ~fr & vis & ~near
        assert act.sum() > 0.2 * n
        for sl in [slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11), slice(11, 14), slice(14, 59)]:
            ww = w["G"][act, sl]
            good, worst = pu.close_bound(got["G"][act, sl], ww, 1e-3, 1e-2 * np.abs(ww).max(), bound[act, sl])
            if not good:  # which Gaussian, and how close its projection's decisions came in each view
                err = np.abs(got["G"][act, sl] - ww) - 1e-3 * (np.abs(ww) + 1e-2 * np.abs(ww).max()) - bound[act, sl]
                i = int(np.nonzero(act)[0][np.unravel_index(np.argmax(err), err.shape)[0]])
                margins = [float(r["fwd"]["proj"]["margin"][i]) for r in w["views"]]
                raise AssertionError((s.n, sl, worst, i, margins, got["G"][i, sl].tolist(), w["G"][i, sl].tolist()))
        # statistics: one visibility per view, norms summed over the views
        assert np.array_equal(got["cnt"], o["cnt"])
        assert o["cnt"].max() >= 2
        clean = (o["cnt"] > 0) & ~amb_rows & ~near
        for key in ("acc_x", "acc_r"):
            good, worst = pu.close(got[key][clean], o[key][clean], 1e-3, 1e-2 * np.abs(o[key][clean]).max())
            assert good, (s.n, key, worst)
        # one Adam step at the scene's counter, from the step's own gradient, at
        # the rates the host set for this iteration (the xyz rate decays each one)
        assert got["step"] == st0["step"] + 1 == o["step"]
        lr = got["lr"].astype(np.float64)
        assert lr[0] == pytest.approx(s.ctrl.lr_xyz_at(k_cmp), rel=1e-6) and np.array_equal(lr[1:], st0["lr"][1:])
        Po, Mo, Vo = (st0[k].astype(np.float64) for k in ("P", "M", "V"))
        Gd = got["G"].astype(np.float64)
        oracle.adam(Po, Gd, Mo, Vo, o["frozen"], lr, got["step"], b1=b1, b2=b2, eps=eps)
        assert np.array_equal(got["P"][fr], st0["P"][fr]) and np.array_equal(got["M"][fr], st0["M"][fr])
        assert np.array_equal(got["V"][fr], st0["V"][fr])
        a = ~fr
        m_scale = b1 * np.abs(st0["M"][a]) + (1 - b1) * np.abs(Gd[a])
        v_scale = b2 * st0["V"][a] + (1 - b2) * Gd[a] ** 2
        assert np.all(np.abs(got["M"][a] - Mo[a]) <= 1e-5 * m_scale + 1e-30)
        assert np.all(np.abs(got["V"][a] - Vo[a]) <= 1e-5 * v_scale + 1e-30)
        grp = np.array([0] * 3 + [1] * 3 + [2] * 4 + [3] + [4] * 3 + [5] * 45)
        bc1, bc2 = 1 - b1 ** got["step"], 1 - b2 ** got["step"]
        step_bound = lr[grp] * (m_scale / bc1) / (np.sqrt(Vo[a] / bc2) + eps)
        spacing = np.spacing(np.abs(st0["P"][a]).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(got["P"][a] - Po[a]) <= 1e-4 * step_bound + 2 * spacing)
