"""Checkpoint / resume: the trainer's state round-trips bit for bit, and a
resumed run continues like the uninterrupted one (up to the rasteriser
backward's atomic reordering)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2504_06716_gb300 import lib, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06716_gb300 import build

    build.build()
    lib.load()


def test_checkpoint_round_trip_and_resume(tmp_path):
    from paper_2504_06716_gb300.schedule import GStaConfig
    from paper_2504_06716_gb300.train import Trainer

    cfg = GStaConfig.tiny()
    scene = synth.tiny_scene()
    a = Trainer(scene, cfg, tile=16)
    while a.k < 60:
        a.iteration()
    path = str(tmp_path / "gsta.ckpt")
    a.save_checkpoint(path)
    saved = torch.load(path, weights_only=False)
    b = Trainer(scene, cfg, tile=16)
    b.load_checkpoint(path)
    st = b.model.state_dict()
    for k in a.model._STATE:
        assert torch.equal(st[k], saved["model"][k]), k
    assert st["n"] == saved["model"]["n"] and st["step_count"] == saved["model"]["step_count"]
    assert b.ctrl.state_dict() == a.ctrl.state_dict() and b.k == a.k == 60 and b.eps0 == a.eps0
    assert b.den_rng.bit_generator.state == a.den_rng.bit_generator.state
    for t in (a, b):
        while t.k < 100:
            t.iteration()
    assert b.model.n == a.model.n and b.model.step_count == a.model.step_count
    pa, pb = a.heldout_psnr(), b.heldout_psnr()
    assert abs(pa - pb) < 0.05, (pa, pb)
    Pa, Pb = a.model.P[: a.model.n, :59], b.model.P[: b.model.n, :59]
    assert (Pa - Pb).abs().max().item() <= 1e-2 * Pa.abs().max().item()
    assert lib.gs_get_device_error() == 0
