"""The training record (``train.JsonlLog``) on host-side stand-ins for the
trainer: cadence, the step a record describes, events written once each."""
import json
from types import SimpleNamespace

import pytest

torch = pytest.importorskip("torch")

from paper_2504_06716_gb300.train import JsonlLog  # noqa: E402


class _Ctrl:
    def lr_xyz_at(self, k):
        return 1e-4 * 0.5 ** (k / 100)


def _trainer():
    model = SimpleNamespace(n=200, n_active=torch.tensor(150))
    view = SimpleNamespace(loss=torch.tensor([0.25]), count=torch.tensor([1234], dtype=torch.int64))
    return SimpleNamespace(k=0, model=model, view=view, events=[], ctrl=_Ctrl())


def test_records_at_cadence_with_events_and_evals(tmp_path):
    p = tmp_path / "log.jsonl"
    log = JsonlLog(str(p), every=3)
    tr = _trainer()
    for it in range(7):  # iterations 0..6 taken
        tr.view.loss = torch.tensor([0.1 * (it + 1)])
        if it == 4:
            tr.events.append((4, "psnr", 31.5))
            tr.events.append((4, "densify", 17))
        tr.k += 1
        log.after_iteration(tr)
    log.evaluation(dict(k=7, wall_s=1.5, heldout_psnr=30.25, n=200, n_active=150))
    log.close()
    recs = [json.loads(line) for line in p.read_text().splitlines()]
    steps = [r for r in recs if "loss" in r]
    assert [r["k"] for r in steps] == [0, 3, 6]
    assert [r["loss"] for r in steps] == pytest.approx([0.1, 0.4, 0.7])
    r = steps[0]
    assert r["n"] == 200 and r["n_active"] == 150 and r["frozen_frac"] == pytest.approx(0.25)
    assert r["entries"] == 1234 and r["lr_xyz"] == pytest.approx(1e-4)
    ev = [r for r in recs if "event" in r]
    assert ev == [dict(k=4, event="psnr", value=31.5), dict(k=4, event="densify", value=17.0)]
    assert recs[-1] == dict(k=7, eval=True, wall_s=1.5, heldout_psnr=30.25, n=200, n_active=150)


def test_rejects_a_zero_cadence(tmp_path):
    with pytest.raises(ValueError):
        JsonlLog(str(tmp_path / "x.jsonl"), every=0)
