"""Learned freeze predictor (not part of the paper).

A 16 -> 64 -> 64 -> 1 MLP with bfloat16 weights and float32 accumulation
that reads a Gaussian's gradient-norm history, opacity, scale, view count
and age and predicts whether the gradient-norm rule of Sec. 3.2.1 (Eqs. 4-6)
will freeze it at one of its next two updates. Applied between updates, it
lets such Gaussians take their siesta earlier; the rule itself stays in
force. All compute runs in the CUDA kernels behind the C ABI
(gs_pred_history, gs_pred_features, gs_mlp_fwd, gs_mlp_grad, gs_mlp_adam,
gs_freeze_apply); this module holds the parameters and the training loop.

Labels: at each rule update u, every Gaussian that is not frozen after the
update is a sample with its features taken just before the update; y = 1 iff
the rule freezes it at update u+1 or u+2 with no reset in between.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import time

import numpy as np
import torch

from . import lib

N_IN, N_H = 16, 64
OFF = dict(W1=0, b1=1024, W2=1088, b2=5184, W3=5248, b3=5312)


class FreezePredictor:
    def __init__(self, device="cuda", seed: int = 0, prior: float = 0.2):
        self.device = torch.device(device)
        g = np.random.default_rng(seed)
        prm = np.zeros(lib.MLP_PARAMS, np.float32)
        prm[OFF["W1"]:OFF["b1"]] = g.uniform(-1, 1, 1024) * np.sqrt(6.0 / N_IN)
        prm[OFF["W2"]:OFF["b2"]] = g.uniform(-1, 1, 4096) * np.sqrt(6.0 / N_H)
        prm[OFF["W3"]:OFF["b3"]] = g.uniform(-1, 1, 64) * np.sqrt(3.0 / N_H)
        prm[OFF["b3"]] = np.log(prior / (1 - prior))
        self.params = torch.from_numpy(prm).to(self.device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, device=self.device)
        self.wb = torch.zeros(lib.MLP_WEIGHTS, dtype=torch.bfloat16, device=self.device)
        lib.gs_mlp_refresh(self.params, self.wb)
        self.step = 0

    def predict(self, X: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        n = X.shape[0]
        p = out if out is not None else torch.empty(n, device=self.device)
        lib.gs_mlp_fwd(n, X, self.wb, self.params, p)
        return p

    def fit(self, X: torch.Tensor, y: torch.Tensor, epochs: int = 400, lr: float = 3e-3, balance: bool = True):
        """Full-batch Adam on the weighted BCE; classes weighted to equal total
        weight when ``balance``."""
        n = X.shape[0]
        pos = float(y.sum().item())
        if balance and 0 < pos < n:
            w = torch.where(y > 0.5, torch.full_like(y, 0.5 / pos), torch.full_like(y, 0.5 / (n - pos)))
            inv = 1.0
        else:
            w, inv = None, 1.0 / n
        losses = []
        for e in range(epochs):
            self.grad.zero_()
            self.loss.zero_()
            lib.gs_mlp_grad(n, X, y, w, inv, self.wb, self.params, self.grad, self.loss)
            self.step += 1
            lib.gs_mlp_adam(self.params, self.grad, self.m, self.v, self.wb, lr, 0.9, 0.999, 1e-8, self.step)
            if e % 50 == 0 or e == epochs - 1:
                losses.append(float(self.loss.item()))
        return losses

    def choose_tau(self, X: torch.Tensor, y: torch.Tensor, precision: float = 0.9) -> float:
        """Decision threshold for held-out samples (X, y): the lowest probability
        at which the predicted positives are still at least `precision`
        correct (the most recall at that precision). Freezing acts on the
        positives, so precision is what a false freeze costs."""
        p = self.predict(X).cpu().numpy()
        yv = y.cpu().numpy() > 0.5
        order = np.argsort(-p, kind="stable")
        prec = np.cumsum(yv[order]) / np.arange(1, len(order) + 1)
        ok = np.nonzero(prec >= precision)[0]
        if len(ok) == 0:
            return 1.0  # nothing reaches the precision: predict no freeze
        return float(np.nextafter(np.float32(p[order[ok[-1]]]), np.float32(-np.inf)))

    def state_dict(self) -> dict:
        return dict(params=self.params.cpu().numpy(), step=self.step)

    def load_state_dict(self, d: dict):
        self.params.copy_(torch.from_numpy(np.asarray(d["params"], np.float32)))
        lib.gs_mlp_refresh(self.params, self.wb)
        self.step = int(d.get("step", 0))


@dataclasses.dataclass
class FreezeLog:
    """Features before each rule update and the frozen map after it."""
    features: list = dataclasses.field(default_factory=list)  # (k, X bf16 on host)
    frozen_after: list = dataclasses.field(default_factory=list)  # (k, uint8 map)
    resets: list = dataclasses.field(default_factory=list)

    def dataset(self):
        """(X, y) over all updates u that have two later updates before any reset."""
        Xs, ys = [], []
        ks = [k for k, _ in self.frozen_after]
        for u in range(len(ks) - 2):
            if any(ks[u] < r <= ks[u + 2] for r in self.resets):
                continue
            _, X = self.features[u]
            f0, f1, f2 = self.frozen_after[u][1], self.frozen_after[u + 1][1], self.frozen_after[u + 2][1]
            cand = f0 == 0
            Xs.append(X[cand])
            ys.append(((f1[cand] == 1) | (f2[cand] == 1)).astype(np.float32))
        if not Xs:
            return None, None
        return torch.cat(Xs), torch.from_numpy(np.concatenate(ys))


def collect(scene, cfg, iters: int, device="cuda", seed: int = 3) -> FreezeLog:
    """Run GSta training on ``scene`` and log the rule's decisions."""
    from .train import Trainer

    tr = Trainer(scene, cfg, device=device, seed=seed)
    tr.enable_predictor_state()
    tr.log = FreezeLog()
    while not tr.finished() and tr.k < iters:
        tr.iteration()
    return tr.log


def evaluate(scene, cfg, predictor: FreezePredictor | None, tau: float, every: int, device="cuda", seed: int = 3,
             shadow: bool = True) -> dict:
    """One GSta run with (or without) the predictor. Reports final loss / PSNR,
    the sum over iterations of the active-Gaussian count (the work freezing
    saves in the backward and the optimiser), and -- with ``shadow`` -- the
    false-freeze rate: the share of predictor-frozen Gaussians whose
    gradient norms, measured by an unmasked backward over the next window,
    would not have passed the rule."""
    from .train import Trainer

    tr = Trainer(scene, cfg, device=device, seed=seed)
    tr.enable_predictor_state()
    tr.shadow = shadow
    if predictor is not None:
        tr.predictor, tr.pred_tau, tr.pred_every = predictor, tau, every
    active_sum = 0
    t0 = time.perf_counter()
    while not tr.finished():
        tr.iteration()
        active_sum += int(tr.model.n_active.item())
    dt = time.perf_counter() - t0
    out = dict(iters=tr.k, active_gaussian_iters=active_sum, heldout_psnr=tr.heldout_psnr(), seconds=dt,
               predicted=tr.pred_count, events=[e for e in tr.events if e[1] != "psnr"])
    if shadow:
        out["false_freeze_rule"] = tr.false_freeze_rate("rule")
        out["false_freeze_pred"] = tr.false_freeze_rate("pred")
        out["shadow_checked"] = dict(tr.shadow_checked)
    return out


FLOPS_PER_ROW = 2 * (N_IN * N_H + N_H * N_H + N_H)  # 10,368: the three layers' multiply-adds
BYTES_PER_ROW = 2 * N_IN + 4  # bf16 features in, float32 probability out


def bench_inference(n: int, reps: int = 20) -> dict:
    """Device time of gs_mlp_fwd on n rows of seeded features (CUDA events on
    the launching stream, after a warm-up; n x 32 B of features exceed L2 for
    n in the millions)."""
    g = torch.Generator(device="cpu").manual_seed(5)
    X = torch.randn((n, N_IN), generator=g).to(torch.bfloat16).cuda()
    pred = FreezePredictor()
    p = torch.empty(n, device="cuda")
    for _ in range(3):
        pred.predict(X, p)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        pred.predict(X, p)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return dict(rows=n, ms=ms, tflops=FLOPS_PER_ROW * n / (ms * 1e-3) / 1e12,
                gbs=BYTES_PER_ROW * n / (ms * 1e-3) / 1e9)


def main():
    from . import synth
    from .schedule import GStaConfig

    ap = argparse.ArgumentParser(description="train the freeze predictor on tiny-scene runs and compare")
    ap.add_argument("--bench-inference", type=int, default=0, help="only time inference on this many rows")
    ap.add_argument("--train-seeds", default="0,1,2,3")
    ap.add_argument("--eval-seed", type=int, default=9)
    ap.add_argument("--val-seeds", default="4,5", help="runs whose logs choose the threshold")
    ap.add_argument("--precision", type=float, default=0.9, help="precision the threshold must reach on them")
    ap.add_argument("--epochs", type=int, default=600)
    ap.add_argument("--balance", type=int, default=1)
    args = ap.parse_args()
    torch.cuda.set_device(0)
    if args.bench_inference:
        print(json.dumps(bench_inference(args.bench_inference)))
        return
    cfg = GStaConfig.tiny()
    logs = []
    for s in [int(x) for x in args.train_seeds.split(",")]:
        logs.append(collect(synth.tiny_scene(seed=s), cfg, cfg.total_iter))
    data = [lg.dataset() for lg in logs]
    X = torch.cat([d[0] for d in data if d[0] is not None])
    y = torch.cat([d[1] for d in data if d[1] is not None]).to(X.device)
    pred = FreezePredictor()
    losses = pred.fit(X, y, epochs=args.epochs, balance=bool(args.balance))
    p = pred.predict(X)
    acc = float(((p > 0.5).float() == y).float().mean().item())
    val = [collect(synth.tiny_scene(seed=int(s)), cfg, cfg.total_iter).dataset() for s in args.val_seeds.split(",")]
    Xv = torch.cat([d[0] for d in val if d[0] is not None])
    yv = torch.cat([d[1] for d in val if d[1] is not None])
    tau = pred.choose_tau(Xv, yv, args.precision)
    scene = synth.tiny_scene(seed=args.eval_seed)
    out = dict(samples=int(X.shape[0]), positives=float(y.mean().item()), train_acc=acc, losses=losses, tau=tau,
               rule_only=evaluate(scene, cfg, None, 1.0, 4), with_predictor=evaluate(scene, cfg, pred, tau, 4))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
