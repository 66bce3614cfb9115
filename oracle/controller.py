"""Host-side schedule of GSta, written out plainly (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Eq. 5 dynamic freeze thresholds, read as eps_k = eps_0 * clamp(0.5 + 1.5 k / K, 0.5, 1.5):
  the literal recursion grows without bound, while Sec. 3.2.1 and Sec. 4.1
  say the thresholds rise with k and stay within [0.5, 1.5] x their initial
  values.
* Sec. 4.1 freeze cadence: the map is updated every 250 iterations inside
  [3000, min(10000, early-stop iteration)), reset every 2000 iterations, and
  not updated for 500 iterations after a reset. Freezing is active only in
  that window, so when it closes at 10000 without an early stop (which
  resets the map itself) the map is reset.
* Eq. 7 early stop: PSNR on the training subset every 1000 iterations; stop
  when the last two PSNR changes are both below 0.2 dB.
* Sec. 3.2.3 plateau schedule on the xyz learning rate: decay 0.75,
  patience 1, threshold read as 1 dB on the PSNR (absolute, mode max).
  Sec. 4.1 says GSta keeps vanilla 3DGS's learning rates except the opacity
  rate, so its xyz rate is vanilla's exponential decay (to 1/100 of the
  start over the iteration budget) times the plateau decays.
* The opacity reset of Sec. 4.1 leaves frozen Gaussians alone: a frozen
  Gaussian takes no parameter change (Sec. 3.2.4); see densify.opacity_reset.
"""
from __future__ import annotations

import dataclasses
import math

from oracle import planted


@dataclasses.dataclass
class ScheduleConfig:
    total_iter: int = 30000
    warmup: int = 3000
    window_end: int = 10000
    every: int = 250
    reset_every: int = 2000
    wait: int = 500
    psnr_every: int = 1000
    eps_psnr: float = 0.2
    finetune_iters: int = 1000
    eps0_xyz: float = 3e-5
    eps0_rgb: float = 1e-4
    lr_decay: float = 0.75
    lr_patience: int = 1
    lr_eps: float = 1.0
    # densification (Sec. 4.1; 3DGS's mechanics): every den_every iterations
    # in (den_from, min(window_end, early stop)), opacity reset every
    # opacity_every in [opacity_every, min(window_end, early stop)]; the plain
    # 3DGS arm densifies until den_until_plain instead.
    den_from: int = 500
    den_every: int = 100
    opacity_every: int = 3000
    den_until_plain: int = 15000
    rgb_every: int = 5  # the diffuse-colour criterion on every fifth densification step (20%)
    eps0_den_xyz: float = 2e-4
    eps0_den_rgb: float = 1e-6


def threshold(eps0: float, k: int, K: int) -> float:
    """Eq. 5 under the clamped-linear reading."""
    f = 0.5 + 1.5 * k / K
    return eps0 * (f if planted(31) else min(1.5, max(0.5, f)))


def freeze_action(k: int, cfg: ScheduleConfig, last_reset: int | None, stop_iter: int | None) -> str | None:
    """What the freeze map does before iteration k: 'update', 'reset', 'clear' (statistics
    only) or None. ``last_reset`` is the iteration of the previous reset, ``stop_iter`` the
    early-stop iteration if it has happened."""
    if k % cfg.every != 0:
        return None
    end = cfg.window_end if stop_iter is None else min(cfg.window_end, stop_iter)
    if stop_iter is None and k == cfg.window_end:
        return "reset"  # the window closes without an early stop: nothing stays frozen
    if k >= end:
        return None
    if k < cfg.warmup:
        return "clear"
    if k % cfg.reset_every == 0:
        return "reset"
    if last_reset is not None and k < last_reset + cfg.wait and not planted(33):
        return "clear"
    return "update"


def early_stop(psnrs: list[float], eps: float) -> bool:
    """Eq. 7: both of the two most recent PSNR changes are below eps (signed changes)."""
    if len(psnrs) < 3:
        return False
    return (psnrs[-1] - psnrs[-2]) < eps and (planted(32) or (psnrs[-2] - psnrs[-3]) < eps)


class Plateau:
    """Decay the learning rate when the PSNR has not improved by more than
    ``eps`` for more than ``patience`` evaluations."""

    def __init__(self, lr: float, decay: float, patience: int, eps: float):
        self.lr, self.decay, self.patience, self.eps = lr, decay, patience, eps
        self.best = -math.inf
        self.bad = 0

    def step(self, psnr: float) -> float:
        if psnr > self.best + self.eps:
            self.best = psnr
            self.bad = 0
        else:
            self.bad += 1
            if self.bad > (0 if planted(36) else self.patience):
                self.lr *= self.decay
                self.bad = 0
        return self.lr


def xyz_rate(k: int, K: int, lr0: float, plateau_factor: float = 1.0, final_ratio: float = 0.01) -> float:
    """xyz learning rate at iteration k: lr0 final_ratio^(min(k, K) / K), vanilla
    3DGS's exponential decay, times the product of the plateau decays so far
    (1 for plain 3DGS)."""
    t = min(max(k, 0), K) / K
    decay = final_ratio ** (1.0 if planted(48) else t)
    return lr0 * decay * plateau_factor


def _den_end(cfg: ScheduleConfig, stop_iter: int | None, plain: bool) -> int:
    if plain:
        return cfg.den_until_plain
    return cfg.window_end if stop_iter is None else min(cfg.window_end, stop_iter)


def densify_due(k: int, cfg: ScheduleConfig, stop_iter: int | None, plain: bool = False) -> bool:
    """Densify and prune after iteration k: k a multiple of den_every in the open
    interval (den_from, end), end = min(window_end, early stop) for GSta."""
    return k % cfg.den_every == 0 and cfg.den_from < k < _den_end(cfg, stop_iter, plain)


def densify_uses_rgb(k: int, cfg: ScheduleConfig) -> bool:
    """Sec. 4.1: the diffuse-colour criterion on 20% of the densification
    steps, read as every fifth one."""
    return (k // cfg.den_every) % cfg.rgb_every == 0


def opacity_reset_due(k: int, cfg: ScheduleConfig, stop_iter: int | None, plain: bool = False) -> bool:
    """Opacity reset after iteration k: k a positive multiple of opacity_every
    up to the densification end (inclusive)."""
    return k > 0 and k % cfg.opacity_every == 0 and k <= _den_end(cfg, stop_iter, plain)


def size_pruning(k: int, cfg: ScheduleConfig) -> bool:
    """Screen / world size pruning once past the first opacity reset."""
    return k > cfg.opacity_every
