"""The schedule defaults of the product (schedule.GStaConfig, the learning
rates of pipeline.default_lrs, the loss weight of the step) and of the
oracle's controller equal the constants the paper prints
(tests/golden/paper_constants.json, each value with its passage). CPU only."""
import json
import os

import pytest

from oracle import controller as C
from paper_2504_06716_gb300 import pipeline
from paper_2504_06716_gb300.schedule import GStaConfig

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def _v(section, key):
    return GOLDEN[section][key][0]


@pytest.mark.parametrize("cfg", [GStaConfig(), C.ScheduleConfig()], ids=["product", "oracle"])
def test_freeze_early_stop_plateau_and_densify_defaults(cfg):
    for key in ("eps0_xyz", "eps0_rgb", "every", "reset_every", "wait", "warmup", "window_end"):
        assert getattr(cfg, key) == _v("freeze", key), key
    assert cfg.eps_psnr == _v("early_stop", "eps_psnr")
    assert cfg.psnr_every == _v("early_stop", "psnr_every")
    assert cfg.lr_decay == _v("learning_rate", "plateau_decay")
    assert cfg.lr_patience == _v("learning_rate", "plateau_patience")
    assert cfg.lr_eps == _v("learning_rate", "plateau_eps")
    for key in ("eps0_den_xyz", "eps0_den_rgb", "den_every", "den_from", "opacity_every"):
        assert getattr(cfg, key) == _v("densify", key), key
    assert 1.0 / cfg.rgb_every == pytest.approx(_v("densify", "rgb_share"))


def test_threshold_scale_stays_within_the_printed_range():
    lo, hi = _v("freeze", "threshold_scale")
    K = 30000
    vals = [C.threshold(1.0, k, K) for k in range(0, K + 1, 250)]
    assert min(vals) == pytest.approx(lo) and max(vals) == pytest.approx(hi)


def test_opacity_rate_and_loss_weight():
    import inspect

    from paper_2504_06716_gb300 import autograd, lib

    assert pipeline.default_lrs(1.0)[3] == _v("learning_rate", "opacity")
    lam = _v("loss", "lambda_ssim")
    # the default SSIM weight of every entry that evaluates Eq. 3
    assert inspect.signature(pipeline.Model.loss).parameters["lam"].default == lam
    assert inspect.signature(autograd.ssim_l1_loss).parameters["lam"].default == lam
    assert inspect.signature(lib.step_args).parameters["lam"].default == lam  # the native training step


def test_trick_gs_defaults():
    cfg = GStaConfig()
    for key in ("prog_start", "prog_until", "blur_until", "sig_fraction", "sig_decay", "mask_from", "mask_until",
                "mask_prune_every"):
        assert getattr(cfg, key) == _v("trick_gs", key), key
    assert list(cfg.sig_iters) == _v("trick_gs", "sig_iters")
