"""The rasteriser backward that resumes behind each tile's last unfrozen splat
(gs_render_fwd_resume / gs_raster_bwd_resume) against the plain calls and the
FP64 oracle.

A frozen Gaussian takes no gradient (Sec. 3.2.4), so the backward needs the
splats behind a tile's last unfrozen one only for the transmittance and the
colour behind it, which the forward records. Checked here:

* the forward's image, T_final and n_last are those of gs_render_fwd_cfg bit
  for bit, and resume_pos is 1 + the position of the last unfrozen entry of
  the tile's walked list (every entry from there to the deepest last
  contributor frozen);
* the gradients equal the oracle's within the parity suite's tolerance
  (1e-3 relative) and the plain backward's within 1e-3 relative (floor 1e-3
  of the largest), with freeze fractions from 0 to 1;
* a map with everything frozen gives no gradient and an empty walk.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2504_06716_gb300 import lib  # noqa: E402

import parity_util as pu  # noqa: E402
import test_gpu_parity as tp  # noqa: E402

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


def _run(st, resume: bool, cfg=None):
    """Forward and backward of one staged view, plain or with the resume record."""
    gcam = st["gcam"]
    n = st["P"].shape[0]
    H, W = gcam.height, gcam.width
    vals = torch.from_numpy(st["vals"].view(np.int32).copy()).to(DEV)
    ranges = torch.from_numpy(st["ranges"].view(np.int32).copy()).to(DEV)
    fr = torch.from_numpy(st["frozen"]).to(DEV)
    img = torch.zeros((3, H, W), device=DEV)
    tf = torch.zeros((H, W), device=DEV)
    nl = torch.zeros((H, W), dtype=torch.int32, device=DEV)
    rs = torch.full((H * W * 4,), float("nan"), device=DEV) if resume else None
    rp = torch.full((gcam.tiles,), -1, dtype=torch.int32, device=DEV) if resume else None
    dl = torch.from_numpy(st["dl"].astype(np.float32)).to(DEV)
    g2 = torch.zeros((n, 12), device=DEV)
    if resume:
        lib.gs_render_fwd_resume(st["spl"], vals, ranges, gcam, cfg, fr, img, tf, nl, rs, rp)
        lib.gs_raster_bwd_resume(st["spl"], vals, ranges, gcam, cfg, tf, nl, dl, fr, rs, rp, g2)
    else:
        lib.gs_render_fwd_cfg(st["spl"], vals, ranges, gcam, cfg, img, tf, nl)
        lib.gs_raster_bwd_cfg(st["spl"], vals, ranges, gcam, cfg, tf, nl, dl, fr, g2)
    torch.cuda.synchronize()
    assert lib.gs_get_device_error() == 0
    out = dict(img=img.cpu().numpy(), tf=tf.cpu().numpy(), nl=nl.cpu().numpy(), g2=g2.cpu().numpy())
    if resume:
        out["rp"] = rp.cpu().numpy()
        out["rs"] = rs.cpu().numpy().reshape(H, W, 4)
    return out


@pytest.mark.parametrize("kind,tile,frac", [("tiny", 16, 0.5), ("ragged", 8, 0.9), ("surface", 8, 0.95),
                                            ("surface", 16, 0.0), ("ragged", 32, 0.7)])
def test_resume_matches_plain_and_oracle(kind, tile, frac):
    st = tp._stage_inputs(kind, tile, frozen_frac=frac, seed=3)
    plain = _run(st, False)
    res = _run(st, True)
    # forward outputs unchanged bit for bit
    assert np.array_equal(res["img"], plain["img"])
    assert np.array_equal(res["tf"], plain["tf"])
    assert np.array_equal(res["nl"], plain["nl"])
    assert np.isfinite(res["rs"]).all()
    # resume_pos: 1 + the last unfrozen entry up to the tile's deepest contributor
    gcam = st["gcam"]
    H, W, T = gcam.height, gcam.width, tile
    tx = (W + T - 1) // T
    nl = plain["nl"]
    frozen, vals, ranges = st["frozen"], st["vals"], st["ranges"]
    skipped = walked = 0
    for t in range(gcam.tiles):
        ty_, tx_ = divmod(t, tx)
        m = int(nl[ty_ * T:(ty_ + 1) * T, tx_ * T:(tx_ + 1) * T].max(initial=0))
        s = int(ranges[t, 0])
        unf = [p for p in range(m) if frozen[vals[s + p]] == 0]
        rp = int(res["rp"][t])
        if unf:
            assert rp >= unf[-1] + 1
            assert frozen[vals[s + rp - 1]] == 0
        assert all(frozen[vals[s + p]] == 1 for p in range(min(rp, m), m))
        walked += m
        skipped += m - min(rp, m)
    if frac == 0.0:
        assert skipped == 0
    # gradients: the plain backward's within float32 rounding, and the oracle's
    fr = frozen == 1
    assert np.all(res["g2"][fr] == 0)
    a = ~fr
    if a.any():
        amb = (st["fw"]["margin"] <= pu.PIXEL_MARGIN).astype(np.uint8)
        want = oracle.render_bwd(st["proj"], st["vals"], st["ranges"], st["ocam"], st["dl"], frozen, amb)
        W9 = pu.grad2d_matrix(want)
        for cols in (slice(0, 2), slice(2, 5), slice(5, 6), slice(6, 9)):
            w = W9[a, cols]
            good, worst = pu.close_bound(res["g2"][a, cols], w, 1e-3, 1e-2 * np.abs(w).max(),
                                         want["amb_abs"][a, cols])
            assert good, (cols, worst)
        # and the plain backward's: two float32 routes to the same transmittance
        # (carried forward, recovered backward by division)
        for cols in (slice(0, 2), slice(2, 5), slice(5, 6), slice(6, 9)):
            w = plain["g2"][a, cols]
            good, worst = pu.close(res["g2"][a, cols], w, 1e-3, 1e-3 * np.abs(w).max())
            assert good, (cols, worst)
    assert np.all(res["g2"][:, 9:] == 0)


def test_resume_with_everything_frozen_is_an_empty_walk():
    st = tp._stage_inputs("surface", 8, frozen_frac=1.0, seed=4)
    assert np.all(st["frozen"] == 1)
    res = _run(st, True)
    assert np.all(res["rp"] == 0)
    assert np.all(res["g2"] == 0)
    plain = _run(st, False)
    assert np.array_equal(res["img"], plain["img"])


def test_resume_buffers_go_together():
    st = tp._stage_inputs("tiny", 16, seed=5)
    gcam = st["gcam"]
    H, W = gcam.height, gcam.width
    vals = torch.from_numpy(st["vals"].view(np.int32).copy()).to(DEV)
    ranges = torch.from_numpy(st["ranges"].view(np.int32).copy()).to(DEV)
    img = torch.zeros((3, H, W), device=DEV)
    tf = torch.zeros((H, W), device=DEV)
    nl = torch.zeros((H, W), dtype=torch.int32, device=DEV)
    rs = torch.zeros(H * W * 4, device=DEV)
    with pytest.raises(lib.GsError):
        lib.gs_render_fwd_resume(st["spl"], vals, ranges, gcam, None, None, img, tf, nl, rs, None)


@pytest.mark.parametrize("tile", [8, 16])
def test_resume_record_is_the_same_for_every_launch_shape(tile):
    """Pixels per thread (the packed two-pixel forward included) and batch size
    change only the launch shape: the record and the forward are bit-identical
    across them, the gradients equal up to atomic reordering."""
    st = tp._stage_inputs("surface", tile, frozen_frac=0.9, seed=6)
    ref = None
    for ppt in (1, 2, 4) if tile >= 16 else (1, 2):
        for batch in (32, 64, 128, 256):
            out = _run(st, True, lib.raster_config(ppt, batch))
            if ref is None:
                ref = out
                continue
            for key in ("img", "tf", "nl", "rp", "rs"):
                assert np.array_equal(out[key], ref[key]), (ppt, batch, key)
            good, worst = pu.close(out["g2"], ref["g2"], 1e-4, 1e-3 * np.abs(ref["g2"]).max())
            assert good, (ppt, batch, worst)
