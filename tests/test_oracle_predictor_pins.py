"""Pins of the oracle's learned freeze predictor (a component the paper does
not have): finite differences, closed forms, hand examples. CPU only."""
import math

import numpy as np
import pytest

O = None


@pytest.fixture(autouse=True)
def _o(orc):
    global O
    O = orc


def _params(seed=0, scale=0.3):
    g = np.random.default_rng(seed)
    return g.normal(0, scale, O.mlp_nparams())


def test_bf16_round_to_nearest_even():
    vals = [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -2.5 - 2 ** -7, 3.14159265, 0.0, -0.0]
    want = [1.0, 1.0, 1.0 + 2 ** -6, 1.0, -2.5, 3.140625, 0.0, -0.0]
    assert list(O.bf16(vals)) == want
    assert O.lib().or_bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6  # tie goes to the even mantissa


def test_mlp_zero_weights_closed_form():
    """With all weights zero, z = b3 for every row: p = sigmoid(b3), the
    loss is the mean BCE of a constant and dL/db3 = mean(p - y)."""
    prm = np.zeros(O.mlp_nparams())
    prm[O.MLP_OFF["b3"]] = 0.7
    prm[O.MLP_OFF["b2"]:O.MLP_OFF["b2"] + 64] = np.linspace(-1, 1, 64)
    X = np.random.default_rng(1).normal(size=(10, 16))
    y = np.array([0, 1] * 5, float)
    p = O.mlp_forward(X, prm, round_bf16=False)
    s = 1 / (1 + math.exp(-0.7))
    assert np.allclose(p, s, rtol=0, atol=1e-15)
    L, g = O.mlp_loss_grad(X, y, prm, round_bf16=False)
    assert L == pytest.approx(np.mean(-y * math.log(s) - (1 - y) * math.log(1 - s)), rel=1e-14)
    assert g[O.MLP_OFF["b3"]] == pytest.approx(np.mean(s - y), rel=1e-14)
    h2 = np.maximum(np.linspace(-1, 1, 64), 0)  # relu(b2): the only nonzero hidden output
    assert np.allclose(g[O.MLP_OFF["W3"]:O.MLP_OFF["W3"] + 64], np.mean(s - y) * h2, atol=1e-15)


@pytest.mark.parametrize("weighted", [False, True])
def test_mlp_gradient_by_central_differences(weighted):
    g = np.random.default_rng(2)
    prm = _params(3)
    X = g.normal(size=(40, 16))
    y = (g.uniform(size=40) < 0.4).astype(float)
    w = g.uniform(0.5, 2.0, 40) if weighted else None
    _, grad = O.mlp_loss_grad(X, y, prm, w=w, round_bf16=False)
    idx = np.concatenate([g.choice(1024, 40, replace=False), 1024 + np.arange(0, 64, 8),
                          1088 + g.choice(4096, 60, replace=False), 5184 + np.arange(0, 64, 8),
                          5248 + np.arange(0, 64, 8), [5312]])
    h = 1e-6
    for k in idx:
        pp, pm = prm.copy(), prm.copy()
        pp[k] += h
        pm[k] -= h
        fd = (O.mlp_loss_grad(X, y, pp, w=w, round_bf16=False)[0] - O.mlp_loss_grad(X, y, pm, w=w, round_bf16=False)[0]) / (2 * h)
        assert grad[k] == pytest.approx(fd, rel=1e-5, abs=1e-10), k


def test_mlp_loss_and_gradient_match_torch_autograd():
    """Without bfloat16 rounding, the forward p = sigmoid(relu(relu(X W1 +
    b1) W2 + b2) . W3 + b3) and the weighted binary cross-entropy's gradient
    over all 5313 parameters against torch autograd in float64."""
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(23)
    n = 57
    X = g.normal(0, 1.5, (n, 16))
    y = (g.uniform(size=n) < 0.4).astype(np.float64)
    w = g.uniform(0.2, 3.0, n)
    prm = _params(5, 0.4)
    t = torch.tensor(prm, dtype=torch.float64, requires_grad=True)
    W1 = t[0:1024].view(16, 64)
    b1 = t[1024:1088]
    W2 = t[1088:5184].view(64, 64)
    b2 = t[5184:5248]
    W3 = t[5248:5312]
    b3 = t[5312]
    Xt = torch.tensor(X)
    z = torch.relu(torch.relu(Xt @ W1 + b1) @ W2 + b2) @ W3 + b3
    wt = torch.tensor(w)
    L = (wt * (torch.nn.functional.softplus(z) - torch.tensor(y) * z)).sum() / wt.sum()
    L.backward()
    p = O.mlp_forward(X, prm, round_bf16=False)
    assert np.allclose(p, torch.sigmoid(z).detach().numpy(), rtol=1e-12, atol=1e-15)
    Lo, go = O.mlp_loss_grad(X, y, prm, w=w, round_bf16=False)
    assert Lo == pytest.approx(float(L.detach()), rel=1e-12)
    gt = t.grad.numpy()
    assert np.allclose(go, gt, rtol=1e-10, atol=1e-14 * np.abs(gt).max())
    assert np.abs(gt[0:1024]).max() > 0 and np.abs(gt[1088:5184]).max() > 0


def test_mlp_rounding_applies_to_inputs_weights_and_first_hidden_layer():
    """Rounding mode equals the unrounded network evaluated on pre-rounded
    inputs and weights, except for the first hidden layer's rounding."""
    prm = _params(4)
    X = np.random.default_rng(5).normal(size=(7, 16))
    r = prm.copy()
    for key, size in (("W1", 1024), ("W2", 4096), ("W3", 64)):
        o = O.MLP_OFF[key]
        r[o:o + size] = O.bf16(prm[o:o + size])
    p_round = O.mlp_forward(X, prm, round_bf16=True)
    p_pre = O.mlp_forward(O.bf16(X), r, round_bf16=False)
    assert np.abs(p_round - p_pre).max() < 2e-2  # only the hidden-layer rounding differs
    assert np.abs(p_round - p_pre).max() > 0


def test_history_hand_example():
    acc_x = np.array([4e-6, 0.0], np.float32)
    acc_r = np.array([2e-8, 0.0], np.float32)
    cnt = np.array([2, 0], np.int32)
    frozen = np.array([0, 1], np.uint8)
    st = np.zeros((2, 12))
    st[:, 8] = [1e-6, 5e-7]
    st[:, 0:4] = [[9, 8, 7, 6], [5, 4, 3, 2]]
    O.pred_history(acc_x, acc_r, cnt, frozen, st)
    # Gaussian 0: EMA 0.5e-6 + 0.5 * 2e-6 = 1.5e-6 (float32 input), history shifted
    assert st[0, 8] == pytest.approx(0.5e-6 + 0.5 * float(np.float32(4e-6)) / 2, rel=1e-12)
    assert list(st[0, 1:4]) == [9, 8, 7] and st[0, 0] == st[0, 8]
    assert st[0, 10] == 2 and st[0, 11] == 0
    # Gaussian 1: not visible, EMA kept, one frozen boundary
    assert st[1, 8] == 5e-7 and st[1, 0] == 5e-7 and list(st[1, 1:4]) == [5, 4, 3]
    assert st[1, 10] == 0 and st[1, 11] == 1


def test_features_hand_example():
    P = np.zeros((1, 59))
    P[0, 3:6] = [-4.0, -3.0, -5.5]
    P[0, 10] = math.log(3.0)  # opacity 0.75
    st = np.zeros((1, 12))
    st[0, 0:4] = [3e-5, 3e-6, 0.0, 3e-3]
    st[0, 4:8] = [1e-4, 1e-5, 1e-3, 1e-40]
    st[0, 10] = math.e - 1
    st[0, 11] = 12
    acc_x = np.array([6e-5], np.float32)
    acc_r = np.array([0.0], np.float32)
    cnt = np.array([2], np.int32)
    X = O.pred_features(P, acc_x, acc_r, cnt, st, 300, 1200, 3e-5, 1e-4)[0]
    want = [0, -1, -8, 2, 0, -1, 1, -8, 0.75, -3.0, -5.5, 1.0, 0.25,
            math.log10(float(np.float32(6e-5)) / 2 / 3e-5), -8, 1.0]
    assert np.allclose(X, want, rtol=0, atol=1e-12)


def test_adam_first_step_moves_by_the_rate():
    prm = _params(6)
    p0 = prm.copy()
    g = np.random.default_rng(7).normal(size=prm.shape)
    m, v = np.zeros_like(prm), np.zeros_like(prm)
    O.mlp_adam(prm, g, m, v, 1e-3, 1, eps=0.0)
    assert np.allclose(prm, p0 - 1e-3 * np.sign(g), rtol=0, atol=1e-15)


def test_freeze_apply_hand_example():
    prob = np.array([0.1, 0.95, 0.5, 0.91, 0.9], np.float32)
    frozen = np.array([1, 0, 0, 0, 0], np.uint8)
    act = O.freeze_apply(prob, 0.9, frozen)
    assert frozen.tolist() == [1, 1, 0, 1, 0]  # strict: 0.9 is not above 0.9
    assert act.tolist() == [2, 4]
