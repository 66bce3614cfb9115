"""The product's host controller (schedule.GStaController) against the
oracle's schedule (oracle/controller.py) over whole runs: freeze actions,
Eq. 5 thresholds, densification and opacity-reset cadence, early stop and
the plateau rate, and the ablation strategy that never freezes. CPU only."""
import pytest

from oracle import controller as C
from paper_2504_06716_gb300.schedule import (FREEZE_CLEAR, FREEZE_RESET, FREEZE_UPDATE, GStaConfig,
                                             GStaController)

NAMES = {FREEZE_UPDATE: "update", FREEZE_RESET: "reset", FREEZE_CLEAR: "clear", None: None}


@pytest.mark.parametrize("stop", [None, 6000, 8750])
@pytest.mark.parametrize("strategy", ["gsta", "none"])
def test_schedule_matches_oracle(stop, strategy):
    cfg = GStaConfig(freeze_strategy=strategy)
    ctrl = GStaController(cfg, lr_xyz=1.6e-4)
    ocfg = C.ScheduleConfig()
    last_reset = None
    for k in range(cfg.total_iter):
        if stop is not None and k == stop:
            ctrl.stop_iter = stop  # as report_psnr sets it; finetuning not entered here
        s = ctrl.stop_iter
        want = C.freeze_action(k, ocfg, last_reset, s)
        if want == "reset":
            last_reset = k
        if strategy == "none" and want == "update":
            want = "clear"
        assert NAMES[ctrl.freeze_mode(k)] == want, k
        assert ctrl.densify_due(k) == C.densify_due(k, ocfg, s), k
        assert ctrl.opacity_reset_due(k) == C.opacity_reset_due(k, ocfg, s), k
        assert ctrl.size_pruning(k) == C.size_pruning(k, ocfg)
        if ctrl.densify_due(k):
            assert ctrl.densify_uses_rgb(k) == C.densify_uses_rgb(k, ocfg)
        ex, er = ctrl.thresholds(k)
        assert ex == pytest.approx(C.threshold(ocfg.eps0_xyz, k, ocfg.total_iter), rel=1e-12)
        assert er == pytest.approx(C.threshold(ocfg.eps0_rgb, k, ocfg.total_iter), rel=1e-12)


def test_plain_schedule_densifies_to_15k():
    cfg = GStaConfig(freezing=False)
    ctrl = GStaController(cfg, lr_xyz=1.6e-4)
    ocfg = C.ScheduleConfig()
    for k in range(cfg.total_iter):
        assert ctrl.freeze_mode(k) is None
        assert ctrl.densify_due(k) == C.densify_due(k, ocfg, None, plain=True), k
        assert ctrl.opacity_reset_due(k) == C.opacity_reset_due(k, ocfg, None, plain=True), k


def test_early_stop_and_plateau_match_oracle():
    seq = [20.0, 24.0, 25.5, 26.1, 26.2, 26.25, 26.3]
    cfg = GStaConfig()
    ctrl = GStaController(cfg, lr_xyz=1.0)
    plateau = C.Plateau(1.0, cfg.lr_decay, cfg.lr_patience, cfg.lr_eps)
    for i, p in enumerate(seq):
        stop = ctrl.report_psnr(1000 * (i + 1), p)
        assert stop == C.early_stop(seq[:i + 1], cfg.eps_psnr)
        assert ctrl.lr_xyz == pytest.approx(plateau.step(p), rel=1e-15)
        if stop:
            assert ctrl.stop_iter == 1000 * (i + 1) and ctrl.finetune_left == cfg.finetune_iters
            break
    else:
        pytest.fail("no early stop")


def test_image_schedules_match_oracle():
    from oracle import image_schedules as IS
    from paper_2504_06716_gb300.schedule import blur_sigma, train_resolution

    cfg = GStaConfig(progressive=True, blur=True)
    for k in list(range(0, 6001, 50)) + [6500, 30000]:
        assert train_resolution(k, cfg, 1237, 822) == IS.size_at(k, 1237, 822)
        assert blur_sigma(k, cfg) == pytest.approx(IS.sigma_at(k), abs=1e-12)
    off = GStaConfig()
    assert train_resolution(0, off, 1237, 822) == (1237, 822) and blur_sigma(0, off) == 0.0


def test_controller_state_round_trip():
    cfg = GStaConfig()
    a = GStaController(cfg, lr_xyz=1.0)
    for i, p in enumerate([20.0, 24.0, 25.5, 26.1]):
        a.report_psnr(1000 * (i + 1), p)
    a.freeze_mode(4000)
    b = GStaController(cfg, lr_xyz=7.0)
    b.load_state_dict(a.state_dict())
    assert b.state_dict() == a.state_dict()
    for k in range(4000, 12001, 250):
        assert a.freeze_mode(k) == b.freeze_mode(k)
    assert a.report_psnr(5000, 26.2) == b.report_psnr(5000, 26.2) and a.lr_xyz == b.lr_xyz


def test_xyz_rate_matches_oracle():
    """GSta: vanilla exponential decay times the plateau decays (Sec. 4.1 keeps
    the vanilla rates); plain 3DGS: the vanilla decay alone."""
    lr0 = 1.6e-4 * 4.4
    g = GStaController(GStaConfig(), lr_xyz=lr0)
    p = GStaController(GStaConfig(freezing=False), lr_xyz=lr0)
    seq = [20.0, 24.0, 24.5, 24.6, 26.0, 26.1, 26.15]
    plateau = C.Plateau(lr0, 0.75, 1, 1.0)
    for i, psnr in enumerate(seq):
        k = 1000 * (i + 1)
        g.report_psnr(k, psnr)
        f = plateau.step(psnr) / lr0
        for kk in (k, k + 500, 30000, 31000):
            assert g.lr_xyz_at(kk) == pytest.approx(C.xyz_rate(kk, 30000, lr0, f), rel=1e-12)
            assert p.lr_xyz_at(kk) == pytest.approx(C.xyz_rate(kk, 30000, lr0), rel=1e-12)
    assert g.lr_xyz < lr0  # a plateau decay happened
