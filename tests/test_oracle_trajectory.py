"""The oracle's steps composed into a short GSta training run (Algorithm 1's
loop on a small seeded scene), checked by the invariants the method states
rather than by stored values:

* a frozen Gaussian gets no gradient, and its parameters and Adam moments
  stay bit-unchanged for as long as it is frozen (Sec. 3.2.4);
* between resets the freeze map only grows (Sec. 3.2.1, Eq. 6); a reset
  clears it (Sec. 4.1);
* the active list is the ascending complement of the freeze map;
* the freeze statistics are the averages of the per-view norms over the
  views in which a Gaussian was visible (Eq. 4);
* training lowers the Eq. 3 loss.

CPU only."""
import numpy as np
import pytest

from paper_2504_06716_gb300 import synth


def _scene(orc):
    g = np.random.default_rng(3)
    n, W, H = 160, 48, 40
    P = np.zeros((n, 59))
    P[:, 0:3] = g.uniform(-0.6, 0.6, (n, 3))
    P[:, 3:6] = g.normal(-2.3, 0.3, (n, 3))
    P[:, 6:10] = g.normal(size=(n, 4))
    P[:, 10] = g.uniform(-1.0, 1.0, n)
    P[:, 11:14] = g.uniform(0.0, 1.0, (n, 3))
    P[:, 14:] = g.normal(0, 0.05, (n, 45))
    P = P.astype(np.float32).astype(np.float64)
    cams = [orc.make_cam(c, tile=16) for c in synth.circle_cameras(4, 3.0, W, H, 60.0)]
    targets = [synth.smooth_image(H, W, 40 + k) for k in range(4)]
    return P, cams, targets


def test_short_gsta_run_keeps_the_freeze_invariants(orc):
    P, cams, targets = _scene(orc)
    n = P.shape[0]
    M, V = np.zeros_like(P), np.zeros_like(P)
    lr = np.array([1.6e-3, 5e-3, 1e-3, 2.5e-2, 2.5e-2, 1.25e-3])
    frozen = np.zeros(n, np.uint8)
    acc_x = np.zeros(n, np.float32)
    acc_r = np.zeros(n, np.float32)
    cnt = np.zeros(n, np.int32)
    seen_x, seen_r, seen_c = np.zeros(n), np.zeros(n), np.zeros(n, np.int64)
    snap = {}  # frozen Gaussian -> (row, m row, v row) when it froze
    first = last = None
    froze_any = False
    for k in range(1, 41):
        v = k % len(cams)
        res = orc.loss_and_grad(P, cams[v], targets[v], frozen=frozen)
        if first is None:
            first = res["loss"]
        last = res["loss"]
        G = res["G"]
        assert np.all(G[frozen != 0] == 0.0)
        vis = res["fwd"]["proj"]["radius"] > 0
        live = vis & (frozen == 0)
        # statistics of the visible, unfrozen Gaussians (Eq. 4's averages)
        acc_x[live] += res["xyz_norm"][live].astype(np.float32)
        acc_r[live] += res["rgb_norm"][live].astype(np.float32)
        cnt[live] += 1
        seen_x[live] += res["xyz_norm"][live]
        seen_r[live] += res["rgb_norm"][live]
        seen_c[live] += 1
        orc.adam(P, G, M, V, frozen, lr, step=k)
        for i, (p0, m0, v0) in snap.items():
            assert np.array_equal(P[i], p0) and np.array_equal(M[i], m0) and np.array_equal(V[i], v0)
        if k % 8 == 0:
            mode = 1 if k == 32 else 0  # a reset at 32
            before = frozen.copy()
            c = cnt.copy()
            ax = np.where(c > 0, acc_x / np.maximum(c, 1).astype(np.float32), 0).astype(np.float32)
            ar = np.where(c > 0, acc_r / np.maximum(c, 1).astype(np.float32), 0).astype(np.float32)
            np.testing.assert_allclose(ax[c > 0], (seen_x / np.maximum(seen_c, 1))[c > 0], rtol=1e-5)
            # thresholds at the 40th percentile of the observed averages: some freeze
            ex = float(np.quantile(ax[c > 0], 0.4)) if np.any(c > 0) else 0.0
            er = float(np.quantile(ar[c > 0], 0.4)) if np.any(c > 0) else 0.0
            act = orc.freeze_update(acc_x, acc_r, cnt, frozen, ex, er, mode)
            if mode == 1:
                assert not frozen.any()
                snap.clear()
            else:
                assert np.all(frozen >= before)  # the map only grows
                new = (before == 0) & (c > 0) & (ax < np.float32(ex)) & (ar < np.float32(er))
                assert np.array_equal(frozen != 0, (before != 0) | new)
                for i in np.nonzero(new)[0]:
                    snap[int(i)] = (P[i].copy(), M[i].copy(), V[i].copy())
                froze_any |= bool(new.any())
            assert np.array_equal(act, np.nonzero(frozen == 0)[0])
            assert not acc_x.any() and not acc_r.any() and not cnt.any()
            seen_x[:], seen_r[:], seen_c[:] = 0, 0, 0
    assert froze_any and len(snap) > 0
    assert last < first
