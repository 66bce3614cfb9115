"""Ablation freeze strategies through the C ABI (gs_freeze_select) against
the oracle (oracle/freeze_variants.py), bit for bit: freeze map, active list,
its length, zeroed statistics; empty, ragged, tie-heavy and full-size
inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import freeze_variants as FV  # noqa: E402
from paper_2504_06716_gb300 import lib  # noqa: E402

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


def _stats(n, seed, ties=False):
    g = np.random.default_rng(seed)
    cnt = g.integers(0, 4, n).astype(np.int32)
    if ties:  # few distinct values: many equal scores
        acc_x = (g.integers(0, 4, n) * 1e-5 * cnt).astype(np.float32)
        acc_r = (g.integers(0, 3, n) * 5e-5 * cnt).astype(np.float32)
    else:
        acc_x = (g.exponential(3e-5, n) * cnt).astype(np.float32)
        acc_r = (g.exponential(1e-4, n) * cnt).astype(np.float32)
    frozen = (g.uniform(0, 1, n) < 0.2).astype(np.uint8)
    u = g.uniform(0, 1, n).astype(np.float32)
    return acc_x, acc_r, cnt, frozen, u


def _run(acc_x, acc_r, cnt, frozen, u, ex, er, strategy, fraction):
    n = frozen.shape[0]
    t = [torch.from_numpy(a.copy()).to(DEV) for a in (acc_x, acc_r, cnt, frozen)]
    ut = torch.from_numpy(u.copy()).to(DEV) if strategy == FV.RANDOM else None
    act = torch.full((max(n, 1),), -1, dtype=torch.int32, device=DEV)
    na = torch.full((1,), -7, dtype=torch.int32, device=DEV)
    ws = torch.full((lib.gs_freeze_select_workspace_bytes(n),), 0x5A, dtype=torch.uint8, device=DEV)  # dirty
    lib.gs_freeze_select(n, *t, float(ex), float(er), strategy, fraction, ut, act, na, ws)
    k = int(na.item())
    return [x.cpu().numpy() for x in t], act.cpu().numpy()[:k], k


@pytest.mark.parametrize("n", [0, 1, 1023, 1025, 200003])
@pytest.mark.parametrize("strategy", [FV.RULE, FV.XYZ, FV.RANDOM, FV.MINGRAD])
def test_freeze_select_bit_exact(n, strategy):
    acc_x, acc_r, cnt, frozen, u = _stats(n, n + 7 * strategy)
    ex, er = np.float32(4e-5), np.float32(1.1e-4)
    (gx, gr, gc, gf), act, k = _run(acc_x, acc_r, cnt, frozen, u, ex, er, strategy, 0.25)
    want_f, want_act = FV.select(acc_x, acc_r, cnt, frozen, ex, er, strategy, 0.25, u)
    assert np.array_equal(gf, want_f)
    assert k == len(want_act) and np.array_equal(act, want_act)
    assert not gx.any() and not gr.any() and not gc.any()
    if strategy == FV.RULE:  # the same decisions as the Eq. 4 update of gs_freeze_update
        f2 = frozen.copy()
        assert np.array_equal(oracle.freeze_update(acc_x.copy(), acc_r.copy(), cnt.copy(), f2, ex, er, 0), act)


@pytest.mark.parametrize("fraction", [0.0, 0.1, 0.25, 1.0])
def test_mingrad_ties_and_fractions(fraction):
    acc_x, acc_r, cnt, frozen, u = _stats(50021, 11, ties=True)
    ex, er = np.float32(2e-5), np.float32(1e-4)
    (_, _, _, gf), act, k = _run(acc_x, acc_r, cnt, frozen, u, ex, er, FV.MINGRAD, fraction)
    want_f, want_act = FV.select(acc_x, acc_r, cnt, frozen, ex, er, FV.MINGRAD, fraction)
    assert np.array_equal(gf, want_f) and np.array_equal(act, want_act)


def test_mingrad_nothing_eligible_and_invalid_args():
    n = 3000
    acc_x, acc_r, cnt, frozen, u = _stats(n, 12)
    cnt[:] = 0
    (_, _, _, gf), act, k = _run(acc_x, acc_r, cnt, frozen, u, 4e-5, 1e-4, FV.MINGRAD, 0.25)
    assert np.array_equal(gf, frozen) and k == int((frozen == 0).sum())
    z = torch.zeros(n, device=DEV)
    zi = torch.zeros(n, dtype=torch.int32, device=DEV)
    zb = torch.zeros(n, dtype=torch.uint8, device=DEV)
    ws = torch.zeros(lib.gs_freeze_select_workspace_bytes(n), dtype=torch.uint8, device=DEV)
    na = torch.zeros(1, dtype=torch.int32, device=DEV)
    for strat, frac, uu, ex in ((FV.RANDOM, 0.25, None, 1.0), (FV.MINGRAD, 1.5, None, 1.0),
                                (FV.MINGRAD, 0.25, None, 0.0), (7, 0.25, None, 1.0)):
        with pytest.raises(lib.GsError):
            lib.gs_freeze_select(n, z, z, zi, zb, ex, 1.0, strat, frac, uu, zi, na, ws)


def test_mingrad_full_size():
    """3M Gaussians (the predictor workload's size), the launch configuration
    training uses."""
    n = 3_000_000
    acc_x, acc_r, cnt, frozen, u = _stats(n, 13)
    ex, er = np.float32(4e-5), np.float32(1.1e-4)
    (_, _, _, gf), act, k = _run(acc_x, acc_r, cnt, frozen, u, ex, er, FV.MINGRAD, 0.25)
    want_f, want_act = FV.select(acc_x, acc_r, cnt, frozen, ex, er, FV.MINGRAD, 0.25)
    assert np.array_equal(gf, want_f) and k == len(want_act) and np.array_equal(act, want_act)
