"""Progressive-resolution targets and blur (Sec. 3.3) through the C ABI
against the oracle (oracle/image_schedules.py): the area resize at the
schedule's sizes and ragged ones, the blur at several widths, the copy below
the blur threshold, a short progressive training run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import image_schedules as IS  # noqa: E402
from paper_2504_06716_gb300 import lib, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06716_gb300 import build

    build.build()
    lib.load()


@pytest.mark.parametrize("W,H,k", [(1237, 822, 0), (1237, 822, 1500), (1237, 822, 3000), (101, 77, None),
                                   (64, 48, 6000)])
def test_resize_area_matches_oracle(W, H, k):
    g = np.random.default_rng(W + H)
    img = g.uniform(0, 1, (3, H, W)).astype(np.float32)
    W2, H2 = IS.size_at(k, W, H) if k is not None else (37, 50)  # (37, 50): shrink x, grow nothing beyond
    src = torch.from_numpy(img).to(DEV)
    dst = torch.full((3, H2, W2), -1.0, device=DEV)
    lib.gs_resize_area(src, 3, W, H, dst, W2, H2)
    want = IS.resize_area(img.astype(np.float64), W2, H2)
    got = dst.cpu().numpy()
    assert np.abs(got - want).max() <= 2e-6


@pytest.mark.parametrize("sigma", [1.0, 0.55, 0.1, 0.05])
def test_blur_matches_oracle(sigma):
    g = np.random.default_rng(int(sigma * 100))
    img = g.uniform(0, 1, (3, 23, 31)).astype(np.float32)
    src = torch.from_numpy(img).to(DEV)
    dst = torch.full_like(src, -1.0)
    lib.gs_blur(src, 3, 31, 23, sigma, dst)
    want = IS.blur(img.astype(np.float64), sigma)
    got = dst.cpu().numpy()
    if sigma < IS.SIGMA_MIN:
        assert np.array_equal(got, img)
    else:
        assert np.abs(got - want).max() <= 2e-6


def test_invalid_arguments():
    x = torch.zeros((3, 4, 5), device=DEV)
    with pytest.raises(lib.GsError):
        lib.gs_resize_area(x, 3, 5, 4, x, 2, 2)  # in place
    with pytest.raises(lib.GsError):
        lib.gs_blur(x, 3, 5, 4, -1.0, torch.zeros_like(x))


def test_progressive_training_runs_and_reaches_full_resolution():
    from paper_2504_06716_gb300.schedule import GStaConfig
    from paper_2504_06716_gb300.train import Trainer

    cfg = GStaConfig.tiny()
    cfg.progressive, cfg.blur, cfg.prog_until, cfg.blur_until = True, True, 60, 60
    tr = Trainer(synth.tiny_scene(), cfg, tile=16)
    sizes = []
    for _ in range(80):
        tr.iteration()
        sizes.append((tr.view.cam.width, tr.view.cam.height))
    assert sizes[0][0] < 128 and sizes[-1] == (128, 128)
    assert all(b[0] >= a[0] for a, b in zip(sizes, sizes[1:]))
    assert lib.gs_get_device_error() == 0
    assert np.isfinite(tr.heldout_psnr())
