"""Parity of the learned freeze predictor's kernels (through the C ABI) with
the FP64 oracle: state update, features, tensor-core inference (also at the
3M-Gaussian size it is applied to), training gradient, Adam, and applying
predictions to the freeze map (bit-exact)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2504_06716_gb300 import lib, synth  # noqa: E402

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


def _state(n, seed):
    g = np.random.default_rng(seed)
    st = np.zeros((n, 12), np.float32)
    st[:, 0:4] = g.exponential(3e-7, (n, 4))
    st[:, 4:8] = g.exponential(4e-9, (n, 4))
    st[:, 8] = st[:, 0]
    st[:, 9] = st[:, 4]
    st[:, 10] = g.integers(0, 500, n)
    st[:, 11] = g.integers(0, 12, n)
    st[g.uniform(size=n) < 0.05, 0:8] = 0.0  # never visible yet
    return st


def _stats(n, seed):
    g = np.random.default_rng(seed)
    cnt = g.integers(0, 6, n).astype(np.int32)
    acc_x = (g.exponential(3e-7, n) * cnt).astype(np.float32)
    acc_r = (g.exponential(4e-9, n) * cnt).astype(np.float32)
    return acc_x, acc_r, cnt


def test_history_update_matches_oracle():
    n = 50001
    st = _state(n, 1)
    acc_x, acc_r, cnt = _stats(n, 2)
    frozen = (np.random.default_rng(3).uniform(size=n) < 0.3).astype(np.uint8)
    t = torch.from_numpy(st.copy()).to(DEV)
    lib.gs_pred_history(n, *(torch.from_numpy(a).to(DEV) for a in (acc_x, acc_r, cnt, frozen)), t)
    want = st.astype(np.float64)
    oracle.pred_history(acc_x, acc_r, cnt, frozen, want)
    assert np.allclose(t.cpu().numpy(), want, rtol=1e-6, atol=0)


def test_features_match_oracle():
    n = 20000
    P = pu.f32(synth.gaussians_surface(n, 4))
    st = _state(n, 5)
    acc_x, acc_r, cnt = _stats(n, 6)
    X = torch.zeros((n, 16), dtype=torch.bfloat16, device=DEV)
    lib.gs_pred_features(n, torch.from_numpy(pu.pack64(P)).to(DEV), *(torch.from_numpy(a).to(DEV) for a in
                                                                      (acc_x, acc_r, cnt, st)),
                         4750, 30000, 2.4e-8, 1.6e-10, X)
    got = X.float().cpu().numpy().astype(np.float64)
    want = oracle.pred_features(P, acc_x, acc_r, cnt, st.astype(np.float64), 4750, 30000, float(np.float32(2.4e-8)),
                                float(np.float32(1.6e-10)))
    # bf16 keeps 8 mantissa bits: within one bf16 ulp of the oracle's value
    assert np.all(np.abs(got - want) <= np.abs(want) * 2 ** -8 + 1e-6)


def _mlp_case(n, seed):
    g = np.random.default_rng(seed)
    prm = g.normal(0, 0.25, oracle.mlp_nparams())
    X = oracle.bf16(g.normal(0, 2, (n, 16)))  # inputs as the features kernel leaves them (bf16)
    wb = np.concatenate([prm[0:1024], prm[1088:5184], prm[5248:5312]])
    return prm, X, wb


def _to_dev(prm, X, wb):
    return (torch.from_numpy(prm.astype(np.float32)).to(DEV), torch.from_numpy(X.astype(np.float32)).to(DEV).to(
        torch.bfloat16), torch.from_numpy(wb.astype(np.float32)).to(DEV).to(torch.bfloat16))


@pytest.mark.parametrize("n", [1, 15, 16, 1000, 4097])
def test_mlp_inference_matches_oracle(n):
    prm, X, wb = _mlp_case(n, 7 + n)
    pt, Xt, wbt = _to_dev(prm, X, wb)
    p = torch.zeros(n, device=DEV)
    lib.gs_mlp_fwd(n, Xt, wbt, pt, p)
    want = oracle.mlp_forward(X, pu.f32(prm), round_bf16=True)
    assert np.abs(p.cpu().numpy() - want).max() < 1e-3


def test_mlp_inference_at_3m_rows_sampled():
    """The size the predictor runs at (3M Gaussians), compared on sampled rows."""
    n = 3_000_000
    prm, X, wb = _mlp_case(n, 11)
    pt, Xt, wbt = _to_dev(prm, X, wb)
    p = torch.zeros(n, device=DEV)
    lib.gs_mlp_fwd(n, Xt, wbt, pt, p)
    rows = np.sort(np.random.default_rng(12).choice(n, 20000, replace=False))
    rows[-1] = n - 1
    want = oracle.mlp_forward(X[rows], pu.f32(prm), round_bf16=True)
    assert np.abs(p.cpu().numpy()[rows] - want).max() < 1e-3


def _clear_of_relu_kinks(X, prm, rel=1e-4):
    """Rows whose hidden pre-activations all sit farther from 0 than float32
    rounding can move them. At a pre-activation within rounding of 0 the ReLU
    gate is decided by the summation order, and a flipped gate changes that
    row's whole contribution to the W1 / W2 gradients; such rows have no
    unique answer in float32, so the gradient case leaves them out."""
    W1 = oracle.bf16(prm[0:1024]).reshape(16, 64)
    W2 = oracle.bf16(prm[1088:5184]).reshape(64, 64)
    a1 = X @ W1 + prm[1024:1088]
    s1 = np.abs(X) @ np.abs(W1) + np.abs(prm[1024:1088])
    h1 = oracle.bf16(np.maximum(a1, 0.0))
    a2 = h1 @ W2 + prm[5184:5248]
    s2 = np.abs(h1) @ np.abs(W2) + np.abs(prm[5184:5248])
    return (np.abs(a1) > rel * s1).all(axis=1) & (np.abs(a2) > rel * s2).all(axis=1)


@pytest.mark.parametrize("weighted", [False, True])
def test_mlp_gradient_matches_oracle(weighted):
    prm, X, wb = _mlp_case(5003, 13)
    prm = pu.f32(prm)
    keep = _clear_of_relu_kinks(X, prm)
    assert keep.mean() > 0.9
    X = X[keep]
    n = X.shape[0]
    g = np.random.default_rng(14)
    y = (g.uniform(size=n) < 0.3).astype(np.float32)
    w = g.uniform(0.2, 3.0, n).astype(np.float32) if weighted else None
    wsum = float(w.astype(np.float64).sum()) if weighted else float(n)
    pt, Xt, wbt = _to_dev(prm, X, wb)
    grad = torch.zeros(oracle.mlp_nparams(), device=DEV)
    loss = torch.zeros(1, device=DEV)
    lib.gs_mlp_grad(n, Xt, torch.from_numpy(y).to(DEV), None if w is None else torch.from_numpy(w).to(DEV),
                    1.0 / wsum, wbt, pt, grad, loss)
    Lw, gw, aw = oracle.mlp_loss_grad(X, y, prm, w=w, round_bf16=True, with_abs=True)
    assert float(loss.item()) == pytest.approx(Lw, rel=1e-4)
    got = grad.cpu().numpy()
    # Each entry is a float32 sum of n per-row terms of both signs; its rounding
    # error scales with sqrt(n) 2^-24 sum|terms| (~4e-6 sum|terms| here), not
    # with |sum|. Allowed: 1e-3 |value| + 2e-5 sum|terms|.
    for key, size in (("W1", 1024), ("b1", 64), ("W2", 4096), ("b2", 64), ("W3", 64), ("b3", 1)):
        o = oracle.MLP_OFF[key]
        good, worst = pu.close_bound(got[o:o + size], gw[o:o + size], 1e-3, 0.0, 2e-5 * aw[o:o + size])
        assert good, (key, worst)


def test_mlp_adam_matches_oracle_and_refreshes_bf16_weights():
    g = np.random.default_rng(15)
    prm = pu.f32(g.normal(0, 0.3, oracle.mlp_nparams()))
    grad = pu.f32(g.normal(0, 1e-2, prm.shape))
    m = pu.f32(g.normal(0, 1e-3, prm.shape))
    v = pu.f32(g.uniform(0, 1e-4, prm.shape))
    t = [torch.from_numpy(a.astype(np.float32)).to(DEV) for a in (prm, grad, m, v)]
    wb = torch.zeros(5184, dtype=torch.bfloat16, device=DEV)
    lr, b1, b2, eps = float(np.float32(1e-3)), float(np.float32(0.9)), float(np.float32(0.999)), float(np.float32(1e-8))
    lib.gs_mlp_adam(t[0], t[1], t[2], t[3], wb, lr, b1, b2, eps, 5)
    po, mo, vo = prm.copy(), m.copy(), v.copy()
    oracle.mlp_adam(po, grad, mo, vo, lr, 5, b1=b1, b2=b2, eps=eps)
    assert np.allclose(t[0].cpu().numpy(), po, rtol=1e-6, atol=1e-7)
    assert np.allclose(t[2].cpu().numpy(), mo, rtol=1e-5, atol=1e-9)
    got_wb = wb.float().cpu().numpy()
    want_wb = oracle.bf16(np.concatenate([t[0].cpu().numpy()[0:1024], t[0].cpu().numpy()[1088:5184],
                                          t[0].cpu().numpy()[5248:5312]]))
    assert np.array_equal(got_wb, want_wb.astype(np.float32))


@pytest.mark.parametrize("n", [0, 1, 3000, 1_000_000])
def test_freeze_apply_bit_exact(n):
    g = np.random.default_rng(n + 16)
    prob = g.uniform(size=n).astype(np.float32)
    frozen = (g.uniform(size=n) < 0.2).astype(np.uint8)
    ft = torch.from_numpy(frozen.copy()).to(DEV)
    act = torch.full((max(n, 1),), -1, dtype=torch.int32, device=DEV)
    na = torch.zeros(1, dtype=torch.int32, device=DEV)
    ws = torch.zeros(lib.gs_freeze_workspace_bytes(n), dtype=torch.uint8, device=DEV)
    lib.gs_freeze_apply(n, torch.from_numpy(prob).to(DEV) if n else torch.zeros(1, device=DEV), 0.8, ft, act, na, ws)
    want = oracle.freeze_apply(prob, 0.8, frozen)
    k = int(na.item())
    assert k == len(want) and np.array_equal(act.cpu().numpy()[:k], want)
    assert np.array_equal(ft.cpu().numpy(), frozen)
