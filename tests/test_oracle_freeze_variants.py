"""Pins of the oracle's ablation freeze strategies (Sec. 5, "Freezing
strategies" and "Gradient information"; Table 3): the rule variant against the
C oracle's Eq. 4 update, hand examples, a brute-force mingrad selection and
the random variant's rate. CPU only."""
import math

import numpy as np
import pytest

from oracle import freeze_variants as FV


def _stats(n, seed, frac_frozen=0.2):
    g = np.random.default_rng(seed)
    cnt = g.integers(0, 4, n).astype(np.int32)
    acc_x = (g.exponential(3e-5, n) * cnt).astype(np.float32)
    acc_r = (g.exponential(1e-4, n) * cnt).astype(np.float32)
    frozen = (g.uniform(0, 1, n) < frac_frozen).astype(np.uint8)
    return acc_x, acc_r, cnt, frozen


def test_rule_strategy_is_the_eq4_update(orc):
    """Strategy RULE takes the same decisions as the C oracle's mode-0 update
    (two separate implementations of Eq. 4)."""
    acc_x, acc_r, cnt, frozen = _stats(5000, 1)
    ex, er = np.float32(4e-5), np.float32(1.1e-4)
    fz, act = FV.select(acc_x, acc_r, cnt, frozen, ex, er, FV.RULE)
    f2 = frozen.copy()
    act2 = orc.freeze_update(acc_x.copy(), acc_r.copy(), cnt.copy(), f2, ex, er, 0)
    assert np.array_equal(fz, f2) and np.array_equal(act, act2)


def test_xyz_only_hand_example():
    """GSta-rgb: the positional criterion alone; cnt = 0 and frozen stay as they are."""
    acc_x = np.array([0.5, 3.0, 0.5, 3.0, 0.0, 2.0], np.float32)
    acc_r = np.array([9.0, 1.0, 0.0, 9.0, 0.0, 0.0], np.float32)
    cnt = np.array([1, 2, 1, 1, 0, 2], np.int32)
    frozen = np.array([0, 0, 0, 1, 0, 0], np.uint8)
    # averages x: 0.5, 1.5, 0.5, 3, -, 1.0 against eps_xyz = 1 (strict)
    fz, act = FV.select(acc_x, acc_r, cnt, frozen, 1.0, 2.0, FV.XYZ)
    assert fz.tolist() == [1, 0, 1, 1, 0, 0] and act.tolist() == [1, 4, 5]
    fz, _ = FV.select(acc_x, acc_r, cnt, frozen, 1.0, 2.0, FV.RULE)  # rgb 9 > 2 keeps Gaussian 0 active
    assert fz.tolist() == [0, 0, 1, 1, 0, 0]


def test_random_uses_the_draws_and_hits_the_rate():
    acc_x, acc_r, cnt, frozen = _stats(8, 2, 0.0)
    cnt[:] = [1, 1, 0, 1, 1, 1, 1, 1]
    frozen[:] = [0, 0, 0, 1, 0, 0, 0, 0]
    u = np.array([0.1, 0.25, 0.0, 0.0, 0.3, 0.2499, 0.9, 0.0], np.float32)
    fz, _ = FV.select(acc_x, acc_r, cnt, frozen, 1.0, 1.0, FV.RANDOM, 0.25, u)
    assert fz.tolist() == [1, 0, 0, 1, 0, 1, 0, 1]  # u < 0.25 among the eligible (2: unseen)
    n = 200000
    acc_x, acc_r, cnt, frozen = _stats(n, 3)
    u = np.random.default_rng(4).uniform(0, 1, n).astype(np.float32)
    fz, _ = FV.select(acc_x, acc_r, cnt, frozen, 1.0, 1.0, FV.RANDOM, 0.25, u)
    elig = (frozen == 0) & (cnt > 0)
    m = elig.sum()
    got = (fz[elig] == 1).sum()
    assert abs(got - 0.25 * m) < 4 * math.sqrt(m * 0.25 * 0.75)


def _mingrad_brute(acc_x, acc_r, cnt, frozen, ex, er, fraction):
    """Python loops: every eligible Gaussian's score in float32, sorted as
    (score, index) tuples, the first floor(fraction m) frozen."""
    f32 = np.float32
    items = []
    for i in range(len(cnt)):
        if frozen[i] or cnt[i] <= 0:
            continue
        ax = f32(acc_x[i]) / f32(cnt[i])
        ar = f32(acc_r[i]) / f32(cnt[i])
        sx, sr = f32(ax / f32(ex)), f32(ar / f32(er))
        items.append((float(sx if sx > sr else sr), i))
    items.sort()
    k = int(math.floor(float(f32(fraction)) * len(items)))
    out = np.array(frozen, np.uint8).copy()
    for _, i in items[:k]:
        out[i] = 1
    return out


@pytest.mark.parametrize("fraction", [0.0, 0.25, 0.5, 1.0])
def test_mingrad_matches_brute_force(fraction):
    acc_x, acc_r, cnt, frozen = _stats(3001, 5)
    ex, er = np.float32(4e-5), np.float32(1.1e-4)
    fz, act = FV.select(acc_x, acc_r, cnt, frozen, ex, er, FV.MINGRAD, fraction)
    want = _mingrad_brute(acc_x, acc_r, cnt, frozen, ex, er, fraction)
    assert np.array_equal(fz, want)
    assert np.array_equal(act, np.nonzero(want == 0)[0])


def test_mingrad_count_order_and_ties():
    """Exactly floor(0.25 m) newly frozen; every one scores no higher than any
    eligible Gaussian left active; equal scores go by index."""
    acc_x, acc_r, cnt, frozen = _stats(10007, 6)
    fz, _ = FV.select(acc_x, acc_r, cnt, frozen, 4e-5, 1.1e-4, FV.MINGRAD, 0.25)
    elig = (frozen == 0) & (cnt > 0)
    new = (fz == 1) & elig
    assert new.sum() == math.floor(0.25 * elig.sum())
    s = FV.mingrad_scores(acc_x, acc_r, cnt, 4e-5, 1.1e-4)
    assert s[new].max() <= s[elig & ~new].min()
    # ties: four equal scores, fraction 0.5 -> the two lowest indices
    acc = np.full(4, 2.0, np.float32)
    fz, act = FV.select(acc, acc, np.ones(4, np.int32), np.zeros(4, np.uint8), 1.0, 1.0, FV.MINGRAD, 0.5)
    assert fz.tolist() == [1, 1, 0, 0] and act.tolist() == [2, 3]


def test_mingrad_reduces_to_the_rule_when_the_cut_matches():
    """If exactly the Gaussians the rule would freeze (score < 1) form the
    lowest floor(fraction m), mingrad and the rule agree."""
    acc_x = np.array([0.1, 0.5, 3.0, 5.0, 0.2, 9.0, 7.0, 4.0], np.float32)
    acc_r = np.array([0.1, 0.2, 0.1, 0.1, 0.3, 0.1, 0.1, 0.1], np.float32)
    cnt = np.ones(8, np.int32)
    frozen = np.zeros(8, np.uint8)
    rule, _ = FV.select(acc_x, acc_r, cnt, frozen, 1.0, 1.0, FV.RULE)
    ming, _ = FV.select(acc_x, acc_r, cnt, frozen, 1.0, 1.0, FV.MINGRAD, 3 / 8)
    assert rule.sum() == 3 and np.array_equal(rule, ming)
