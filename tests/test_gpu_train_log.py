"""A short training run through ``train.run`` with the JSON-lines record on
(plain arm: it ends at the iteration count; no freezing, no densification yet)."""
import json
import math

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_short_run_writes_the_training_record(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06716_gb300 import build, lib, train

    build.build()
    lib.load()
    p = tmp_path / "train.jsonl"
    args = train.parser().parse_args(["--arm", "plain", "--n-init", "3000", "--n-gt", "4000", "--views", "16",
                                      "--width", "160", "--height", "120", "--iters", "40", "--eval-every", "20",
                                      "--tune-after", "0", "--log-jsonl", str(p), "--log-every", "10"])
    out = train.run(args)
    assert out["iters"] == 40 and out["device_flags"] == 0
    recs = [json.loads(line) for line in p.read_text().splitlines()]
    steps = [r for r in recs if "loss" in r]
    assert [r["k"] for r in steps] == [0, 10, 20, 30]
    for r in steps:
        assert math.isfinite(r["loss"]) and 0.0 < r["loss"] < 2.0
        assert r["n"] == 3000 and r["n_active"] == 3000 and r["frozen_frac"] == 0.0 and r["entries"] > 0
    evals = [r for r in recs if r.get("eval")]
    assert [r["k"] for r in evals] == [20, 40]
    assert [r["heldout_psnr"] for r in evals] == pytest.approx([e["heldout_psnr"] for e in out["evals"]])
