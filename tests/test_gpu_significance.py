"""Significance pruning (Sec. 3.3, after LightGaussian) through the C ABI
against the oracle (oracle/significance.py): per-Gaussian hit counts of a
view, the scores' selection, the pruning pass and a short training run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import significance as S  # noqa: E402
from paper_2504_06716_gb300 import lib, pipeline, synth  # noqa: E402

import parity_util as pu  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06716_gb300 import build

    build.build()
    oracle.build()
    lib.load()


def test_hit_counts_match_oracle():
    P = synth.gaussians_uniform(1733, 17)
    P[:, 3:6] += 0.8
    P = pu.f32(P)
    n = P.shape[0]
    cam = synth.circle_cameras(3, 3.5, 100, 75, 55.0)[1]
    ocam, gcam = pu.cameras(cam, tile=8)
    proj = oracle.project(P, ocam)
    rec = pu.records_from_oracle(proj)
    vals, ranges = oracle.sort_records(rec, ocam.width, ocam.height, ocam.tile)
    fw = oracle.render(proj, vals, ranges, ocam)
    want = S.hit_counts(proj, vals, ranges.reshape(-1, 2), ocam, n)
    spl = torch.from_numpy(rec).to(DEV)
    vt = torch.from_numpy(vals.view(np.int32).copy()).to(DEV)
    rt = torch.from_numpy(ranges.view(np.int32).copy()).to(DEV)
    img = torch.zeros((3, 75, 100), device=DEV)
    tf = torch.zeros((75, 100), device=DEV)
    nl = torch.zeros((75, 100), dtype=torch.int32, device=DEV)
    lib.gs_render_fwd(spl, vt, rt, gcam, img, tf, nl)
    hits = torch.zeros(n, dtype=torch.int32, device=DEV)
    lib.gs_hit_counts(spl, vt, rt, gcam, nl, hits)
    lib.gs_hit_counts(spl, vt, rt, gcam, nl, hits)  # adds: twice the view
    got = hits.cpu().numpy().astype(np.int64)
    assert got.sum() > 10000
    amb = int((fw["margin"] <= pu.PIXEL_MARGIN).sum())  # pixels whose decisions may flip
    diff = np.abs(got - 2 * want)
    assert diff.sum() <= 2 * 4 * amb, (diff.sum(), amb)
    assert (diff == 0).mean() > 0.99


@pytest.mark.parametrize("n,fraction", [(50021, 0.75), (50021, 0.6), (1, 0.75), (4099, 0.0)])
def test_significance_marks_match_oracle(n, fraction):
    g = np.random.default_rng(n)
    P = np.zeros((n, 59))
    P[:, 3:6] = g.normal(-2.0, 0.7, (n, 3))
    P[:, 10] = g.normal(0.0, 2.0, n)
    P = pu.f32(P)
    hits = g.integers(0, 500, n)
    want_s = S.scores(P, hits)
    want = S.mark(want_s, fraction)
    m = pipeline.Model(P, device=DEV)
    ht = torch.from_numpy(hits.astype(np.int32)).to(DEV)
    got = m.significance_mark(ht, fraction).cpu().numpy()[:n]
    k = int(np.floor(np.float32(fraction) * n))
    assert got.sum() == k == want.sum()
    if k:
        cut = np.sort(want_s)[k - 1]
        near = np.abs(want_s - cut) <= 1e-5 * max(cut, 1e-30)
        assert np.array_equal(got[~near], want[~near])


def test_prune_marked_removes_exactly_the_marked():
    P = pu.f32(synth.gaussians_uniform(3000, 3))
    m = pipeline.Model(P, device=DEV)
    mark = torch.from_numpy((np.arange(3000) % 4 == 1).astype(np.uint8)).to(DEV)
    res = m.prune_marked(mark, np.random.default_rng(0))
    keep = np.arange(3000) % 4 != 1
    assert res["n"] == keep.sum()
    assert np.array_equal(m.P[: res["n"], :59].cpu().numpy(), P[keep].astype(np.float32))


def test_training_with_significance_pruning():
    from paper_2504_06716_gb300.schedule import GStaConfig
    from paper_2504_06716_gb300.train import Trainer

    cfg = GStaConfig.tiny()
    cfg.significance, cfg.sig_iters = True, (30, 60)
    tr = Trainer(synth.tiny_scene(), cfg, tile=16)
    n0 = tr.model.n
    while tr.k < 70:
        tr.iteration()
    ev = [e for e in tr.events if e[1] == "significance_prune"]
    assert len(ev) == 2
    assert ev[0][2] == n0 - int(np.floor(np.float32(0.75) * n0))
    assert lib.gs_get_device_error() == 0
    assert np.isfinite(tr.heldout_psnr())
