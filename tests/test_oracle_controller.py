"""Pins of the oracle's host-side schedule against hand-derived values
(tests/golden/controller_schedule.json, each group citing the passage it
follows). CPU only."""
import json
import os

import pytest

from oracle import controller as C

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "controller_schedule.json")))


def test_threshold_sequence():
    t = GOLD["threshold"]
    for k, want in t["cases"]:
        assert C.threshold(t["eps0"], k, t["K"]) == pytest.approx(want, rel=1e-12)


def _replay(cases, stop_iter):
    cfg = C.ScheduleConfig()
    last_reset = None
    for k in range(0, max(k for k, _ in cases) + 1):
        a = C.freeze_action(k, cfg, last_reset, stop_iter)
        if a == "reset":
            last_reset = k
        yield k, a


@pytest.mark.parametrize("name,stop", [("no_stop", None), ("stop_at_7000", 7000)])
def test_freeze_cadence(name, stop):
    want = dict((k, a) for k, a in GOLD["freeze_action"][name])
    got = dict(_replay(GOLD["freeze_action"][name], stop))
    for k, a in want.items():
        assert got[k] == a, k


def test_early_stop_rule():
    for psnrs, want in GOLD["early_stop"]:
        assert C.early_stop(psnrs, 0.2) is want, psnrs


def test_plateau_schedule():
    p = GOLD["plateau"]
    s = C.Plateau(p["lr0"], 0.75, 1, 1.0)
    assert [s.step(v) for v in p["psnrs"]] == pytest.approx(p["lrs"])


def test_densification_cadence_hand_values():
    cfg = C.ScheduleConfig()
    due = [k for k in range(0, 12001) if C.densify_due(k, cfg, None)]
    assert due[0] == 600 and due[-1] == 9900 and len(due) == 94  # (500, 10000), every 100
    assert [k for k in range(0, 12001) if C.densify_due(k, cfg, 7000)][-1] == 6900  # early stop ends it
    assert [k for k in range(0, 20001) if C.densify_due(k, cfg, None, plain=True)][-1] == 14900
    assert [k for k in range(0, 12001) if C.opacity_reset_due(k, cfg, None)] == [3000, 6000, 9000]
    assert [k for k in range(0, 12001) if C.opacity_reset_due(k, cfg, 6000)] == [3000, 6000]
    rgb = [k for k in due if C.densify_uses_rgb(k, cfg)]
    assert rgb[:3] == [1000, 1500, 2000] and abs(len(rgb) / len(due) - 0.2) < 0.02
    assert not C.size_pruning(3000, cfg) and C.size_pruning(3100, cfg)
    assert C.threshold(cfg.eps0_den_xyz, 0, 30000) == pytest.approx(1e-4)


def test_xyz_rate_hand_values():
    x = GOLD["xyz_rate"]
    for k, factor, want in x["cases"]:
        assert C.xyz_rate(k, x["K"], x["lr0"], factor) == pytest.approx(want, rel=1e-12), k
