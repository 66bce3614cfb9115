"""Pins of the oracle's densification / pruning / opacity reset (3DGS rules
with the paper's thresholds and cadence, Sec. 4.1), on the CPU."""
import math

import numpy as np
import pytest

from oracle import densify as D


def _prm(**kw):
    base = dict(eps_xyz=2e-4, eps_rgb=1e-6, use_rgb=False, log_clone_max=math.log(0.01 * 4.4),
                logit_min_opacity=D.logit(0.005), prune_big=False, max_screen_radius=20,
                log_max_world=math.log(0.1 * 4.4), log_split_div=math.log(1.6))
    base.update(kw)
    return D.DensifyParams(**base)


def _gauss(mean, log_s, logit, quat=(1.0, 0.0, 0.0, 0.0)):
    p = np.zeros(59)
    p[0:3] = mean
    p[3:6] = log_s
    p[6:10] = quat
    p[10] = logit
    p[11:14] = (0.1, 0.2, 0.3)
    return np.asarray(p, np.float32).astype(np.float64)


def test_hand_example_clone_split_prune_and_order():
    small, large = math.log(0.01), math.log(0.2)  # 0.01 < 0.044 clones, 0.2 splits
    P = np.stack([
        _gauss((0, 0, 0), (small,) * 3, 2.0),          # 0: candidate, small -> cloned
        _gauss((1, 2, 3), (large, small, small), 2.0),  # 1: candidate, large -> split
        _gauss((0, 1, 0), (small,) * 3, -8.0),          # 2: opacity 3e-4 < 0.005 -> pruned
        _gauss((0, 0, 1), (small,) * 3, 1.0),           # 3: below the threshold -> kept
        _gauss((2, 0, 0), (small,) * 3, 1.0),           # 4: never seen (cnt 0) -> kept
        _gauss((3, 0, 0), (small,) * 3, -9.0),          # 5: candidate but transparent: clone and original pruned
    ])
    acc = np.array([3e-3, 3e-3, 3e-3, 1e-4, 0.0, 3e-3], np.float32)
    cnt = np.array([5, 5, 5, 5, 0, 5])
    z = np.array([[[1.0, 0.0, 0.0], [0.0, -1.0, 2.0]]])
    out = D.densify(P, acc, np.zeros(6, np.float32), cnt, np.zeros(6, int), _prm(), z)
    assert out["src"].tolist() == [0, 3, 4, 0, 1, 1]
    assert out["kind"].tolist() == [0, 0, 0, 1, 2, 3]
    assert out["counts"] == dict(kept=3, clones=1, children=2, splits=1)
    np.testing.assert_array_equal(out["P"][3], P[0])  # the clone is an exact copy
    s = np.exp(P[1, 3:6])
    np.testing.assert_allclose(out["P"][4, 0:3], P[1, 0:3] + s * z[0, 0], rtol=0, atol=1e-12)  # identity rotation
    np.testing.assert_allclose(out["P"][5, 0:3], P[1, 0:3] + s * z[0, 1], rtol=0, atol=1e-12)
    np.testing.assert_allclose(np.exp(out["P"][4, 3:6]), s / 1.6, rtol=1e-6)
    np.testing.assert_array_equal(out["P"][4, 6:59], P[1, 6:59])


def test_rgb_criterion_only_on_rgb_steps():
    P = np.stack([_gauss((0, 0, 0), (math.log(0.01),) * 3, 2.0)])
    acc_x, acc_r, cnt = np.array([1e-5], np.float32), np.array([1e-5], np.float32), np.array([2])
    off = D.densify(P, acc_x, acc_r, cnt, [0], _prm(use_rgb=False), np.zeros((0, 2, 3)))
    on = D.densify(P, acc_x, acc_r, cnt, [0], _prm(use_rgb=True), np.zeros((0, 2, 3)))
    assert off["counts"]["clones"] == 0 and on["counts"]["clones"] == 1


def test_size_pruning_only_when_enabled():
    P = np.stack([_gauss((0, 0, 0), (math.log(0.5),) * 3, 2.0),   # 0.5 > 0.44: too big in the world
                  _gauss((0, 0, 0), (math.log(0.01),) * 3, 2.0)])  # fine, but 25 px on screen
    args = (np.zeros(2, np.float32), np.zeros(2, np.float32), np.zeros(2), np.array([3, 25]))
    assert D.densify(P, *args, _prm(prune_big=False), np.zeros((0, 2, 3)))["src"].tolist() == [0, 1]
    assert D.densify(P, *args, _prm(prune_big=True), np.zeros((0, 2, 3)))["src"].tolist() == []


def test_children_follow_the_gaussian_covariance():
    """Children offsets of a rotated anisotropic Gaussian: covariance
    R diag(s^2) R^T (checked statistically; a wrong rotation convention or
    s instead of s^2 fails)."""
    g = np.random.default_rng(0)
    q = np.array([0.8, 0.3, -0.4, 0.2])
    log_s = np.log([0.3, 0.1, 0.05])
    m = 4000
    P = np.stack([_gauss((0.5, -1.0, 2.0), log_s, 2.0, q)] * m)
    acc, cnt = np.full(m, 1e-2, np.float32), np.full(m, 1)
    z = g.standard_normal((m, 2, 3))
    out = D.densify(P, acc, acc, cnt, np.zeros(m, int), _prm(), z)
    off = out["P"][:, 0:3] - P[0, 0:3]
    assert out["counts"]["children"] == 2 * m
    qn = q / np.linalg.norm(q)
    w, x, y, zq = qn
    R = np.array([[1 - 2 * (y * y + zq * zq), 2 * (x * y - w * zq), 2 * (x * zq + w * y)],
                  [2 * (x * y + w * zq), 1 - 2 * (x * x + zq * zq), 2 * (y * zq - w * x)],
                  [2 * (x * zq - w * y), 2 * (y * zq + w * x), 1 - 2 * (x * x + y * y)]])
    want = R @ np.diag(np.exp(2 * np.asarray(P[0, 3:6]))) @ R.T
    got = np.cov(off.T)
    assert np.abs(got - want).max() < 0.05 * np.abs(want).max()
    # the exact offsets for the draws given
    np.testing.assert_allclose(off[0], R @ (np.exp(P[0, 3:6]) * z[0, 0]), atol=1e-12)


def test_opacity_reset_caps_and_clears_moments():
    P = np.zeros((3, 59), np.float32)
    P[:, 10] = [-6.0, -4.0, 3.0]
    M, V = np.ones((3, 59), np.float32), np.ones((3, 59), np.float32)
    cap = D.logit(0.01)
    D.opacity_reset(P, M, V, cap)
    assert P[:, 10].tolist() == [-6.0, np.float32(cap), np.float32(cap)]
    assert not M[:, 10].any() and not V[:, 10].any()
    assert M[:, 9].all() and V[:, 11].all()
    # frozen Gaussians keep opacity and moments
    P2 = np.zeros((3, 59), np.float32)
    P2[:, 10] = [-6.0, -4.0, 3.0]
    M2, V2 = np.ones((3, 59), np.float32), np.ones((3, 59), np.float32)
    D.opacity_reset(P2, M2, V2, cap, frozen=np.array([0, 1, 1], np.uint8))
    assert P2[:, 10].tolist() == [-6.0, -4.0, 3.0] and M2[1:, 10].all() and V2[1:, 10].all()


def test_carry_keeps_survivors_and_zeroes_new():
    vals = np.array([[1.0], [2.0], [3.0]])
    out = D.carry(vals, np.array([0, 2, 0, 1, 1]), np.array([0, 0, 1, 2, 3]))
    assert out.ravel().tolist() == [1.0, 3.0, 0.0, 0.0, 0.0]
