"""What the learned freeze predictor buys on the tiny-scene workload.

The predictor is trained (by its own CUDA kernels) on the freeze decisions
the gradient-norm rule logs over four tiny-scene runs, then a held-out scene
is trained twice: with the rule alone and with the predictor applied every 4
iterations (tau = 0.9). Asserted: the predictor run does measurably less
work -- at least 5% fewer active-Gaussian iterations, the quantity freezing
saves in the backward and the optimiser -- for at most 1 dB of held-out PSNR,
and its false-freeze rate (the share of Gaussians it froze whose unmasked
gradient norms over the following window would not have passed the rule) is
measured and reported next to the rule's own.
"""
import json

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06716_gb300 import build, lib

    build.build()
    lib.load()


def test_predictor_saves_work_on_a_held_out_scene():
    from paper_2504_06716_gb300 import synth
    from paper_2504_06716_gb300.predictor import FreezePredictor, collect, evaluate
    from paper_2504_06716_gb300.schedule import GStaConfig

    cfg = GStaConfig.tiny()
    logs = [collect(synth.tiny_scene(seed=s), cfg, cfg.total_iter) for s in (0, 1, 2, 3)]
    data = [lg.dataset() for lg in logs]
    X = torch.cat([d[0] for d in data if d[0] is not None])
    y = torch.cat([d[1] for d in data if d[1] is not None]).to(X.device)
    assert 0.02 < float(y.mean()) < 0.98  # both classes present
    pred = FreezePredictor()
    losses = pred.fit(X, y, epochs=600)
    assert losses[-1] < losses[0]
    scene = synth.tiny_scene(seed=9)
    rule = evaluate(scene, cfg, None, 1.0, 4)
    withp = evaluate(scene, cfg, pred, 0.9, 4)
    print(json.dumps(dict(samples=int(X.shape[0]), rule=rule, predictor=withp), default=str))
    assert withp["predicted"] > 0
    assert withp["active_gaussian_iters"] <= 0.95 * rule["active_gaussian_iters"]
    assert withp["heldout_psnr"] >= rule["heldout_psnr"] - 1.0
    ff = withp["false_freeze_pred"]
    assert ff is not None and 0.0 <= ff <= 1.0
