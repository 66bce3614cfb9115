"""Host-side GSta controller: freeze thresholds, freeze cadence, early stop
and the plateau learning-rate schedule (Algorithm 1's scalar logic).

Readings of the paper taken here:
* Eq. 5 -- thresholds rise linearly with the iteration and stay within
  [0.5, 1.5] x their initial values (Sec. 3.2.1, Sec. 4.1):
  eps_k = eps_0 * min(1.5, max(0.5, 0.5 + 1.5 k / K)).
* Sec. 4.1 -- the map is updated every 250 iterations inside
  [3000, min(10000, early-stop iteration)); reset every 2000 iterations and
  left alone for 500 iterations after a reset; the gradient statistics are
  restarted at every 250-iteration boundary, so each update averages the
  iterations since the previous boundary. Freezing is active only in that
  window: if it closes at 10000 without an early stop, the map is reset.
* Eq. 7 -- PSNR of a fixed training subset every 1000 iterations while the
  freezing phase lasts; stop when the last two changes are both < 0.2 dB;
  then all Gaussians are unfrozen for a finetuning stage of K_f iterations,
  after which training ends.
* Sec. 3.2.3 -- the xyz learning rate decays by 0.75 when the PSNR has not
  risen by more than 1 dB for more than one evaluation; Sec. 4.1 keeps the
  vanilla rates, so these decays multiply vanilla 3DGS's exponential decay
  of the xyz rate (to 1/100 over the iteration budget).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FREEZE_UPDATE, FREEZE_RESET, FREEZE_CLEAR = 0, 1, 2


@dataclasses.dataclass
class GStaConfig:
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
    freezing: bool = True  # False: plain 3DGS training (no freezing, no early stop)
    # plain 3DGS decays the xyz rate exponentially to 1/100 over the run
    # (Sec. 3.2.3 describes the vanilla decay that GSta's plateau schedule replaces)
    plain_lr_final_ratio: float = 0.01
    # densification (Sec. 4.1; clone / split / prune are 3DGS's): every den_every
    # iterations in (den_from, min(window_end, early stop)) -- den_until_plain
    # for plain 3DGS -- with thresholds eps0_den scaled like Eq. 5; the
    # diffuse-colour criterion on every rgb_every-th step (the paper's 20%);
    # opacity reset every opacity_every iterations up to the same end.
    densify: bool = True
    den_from: int = 500
    den_every: int = 100
    den_until_plain: int = 15000
    rgb_every: int = 5
    opacity_every: int = 3000
    eps0_den_xyz: float = 2e-4
    eps0_den_rgb: float = 1e-6
    percent_dense: float = 0.01     # of the scene extent: largest scale that clones
    min_opacity: float = 0.005
    # 3DGS's screen-size rule (20 px) reads the window's largest screen radii,
    # which 3DGS clears in its clone / split step before the prune test reads
    # them, so in 3DGS as run it removes nothing: None keeps it off (an int
    # turns it on with that many pixels).
    max_screen_radius: int | None = None
    max_world_frac: float = 0.1     # of the scene extent
    split_div: float = 1.6
    # freeze strategy of the ablation (Sec. 5, Table 3): "gsta" the Eq. 4 rule;
    # "xyz" the rule on positional gradients only (GSta-rgb); "random" /
    # "mingrad" freeze freeze_fraction of the eligible Gaussians at random / with
    # the lowest gradients; "none" keeps GSta's schedule, early stop and LR
    # plateau but never freezes (GSta-freezing).
    freeze_strategy: str = "gsta"
    freeze_fraction: float = 0.25
    # finetune with the absolute-value opacity activation instead of the
    # sigmoid (Sec. 4.1, the trick taken from Taming 3DGS)
    abs_opacity_finetune: bool = True
    # the opacity's Adam moments at that switch: "rescale" carries them over
    # to the new parameterisation, "zero" restarts them
    abs_opacity_moments: str = "rescale"
    # Trick-GS image-space schedules (Sec. 3.3, Sec. 4.1; off in plain GSta):
    # train on the area-averaged target at scale prog_start rising by a cosine
    # to full resolution at prog_until; blur the target with a 5x5 Gaussian
    # whose sigma (pixels) falls by a cosine from blur_sigma0 to 0 at blur_until
    progressive: bool = False
    prog_start: float = 0.175
    prog_until: int = 6000
    blur: bool = False
    blur_sigma0: float = 1.0
    blur_until: int = 6000
    # Trick-GS volume masks (Sec. 3.3 "Pruning with Volume Masking"; Sec. 4.1:
    # learned from 1K to 10K, masked Gaussians pruned every 1K): a mask logit
    # per Gaussian (float 59 of its row), hard mask 1[sigmoid(m) > 0.01] on
    # opacity and scales, straight-through gradient, loss term
    # mask_lambda * mean sigmoid(m); rate, weight and start value are the
    # compact-3DGS method's defaults (readings)
    volume_mask: bool = False
    mask_init: float = 2.0
    mask_lr: float = 0.01
    mask_lambda: float = 5e-4
    mask_from: int = 1000
    mask_until: int = 10000
    mask_prune_every: int = 1000
    # Trick-GS significance pruning (Sec. 3.3, after LightGaussian; Sec. 4.1):
    # at sig_iters, remove the least significant sig_fraction of the Gaussians
    # (times sig_decay per earlier pruning); score = hits * opacity *
    # (volume / 90th-percentile volume)^sig_beta over the training views
    significance: bool = False
    sig_iters: tuple = (4000, 7000)
    sig_fraction: float = 0.75
    sig_decay: float = 0.8
    sig_beta: float = 0.1
    sig_quantile: float = 0.9
    # opacity learning rate under |x|: "slope" scales the training rate by the
    # mean o (1 - o) at the switch, so that an Adam step moves opacities by
    # as much on average as it did through the sigmoid; None keeps 0.025; a
    # number sets it
    abs_opacity_lr: float | str | None = "slope"
    # Eq. 7 on (False: PSNR is still checked, for the plateau rate, but the
    # run never stops early and trains to total_iter)
    early_stop: bool = True
    # reset the map when the freezing window closes at window_end without an
    # early stop (False: the Gaussians frozen last stay frozen to total_iter)
    window_end_reset: bool = True
    # what the opacity reset does to a frozen Gaussian: "skip" leaves it
    # untouched (a frozen Gaussian takes no parameter change, Sec. 3.2.4);
    # "reset" caps its opacity like every other's (3DGS); "unfreeze" caps
    # every opacity and resets the map
    opacity_reset_frozen: str = "skip"
    # Sec. 4.1: GSta keeps vanilla 3DGS's learning rates (opacity aside), so
    # the plateau decays of Sec. 3.2.3 multiply the vanilla exponential decay
    # of the xyz rate; False: they replace it (a constant rate between decays)
    plateau_on_vanilla: bool = True
    # vanilla 3DGS's opacity rate for the plain arm (Sec. 4.1 sets GSta's to
    # 0.025 "except" the vanilla one)
    plain_opacity_lr: float = 0.05

    @staticmethod
    def tiny() -> "GStaConfig":
        """The schedule scaled to a 200-iteration run (no densification)."""
        return GStaConfig(total_iter=200, warmup=20, window_end=150, every=10, reset_every=80, wait=20, psnr_every=20,
                          finetune_iters=20, densify=False)


class GStaController:
    def __init__(self, cfg: GStaConfig, lr_xyz: float):
        self.cfg = cfg
        self.lr_xyz = lr_xyz
        self._best = float("-inf")
        self._bad = 0
        self.psnrs: list[float] = []
        self.last_reset: int | None = None
        self.stop_iter: int | None = None
        self.finetune_left: int | None = None

    def state_dict(self) -> dict:
        return dict(lr_xyz=self.lr_xyz, best=self._best, bad=self._bad, psnrs=list(self.psnrs),
                    last_reset=self.last_reset, stop_iter=self.stop_iter, finetune_left=self.finetune_left)

    def load_state_dict(self, st: dict):
        self.lr_xyz, self._best, self._bad = st["lr_xyz"], st["best"], st["bad"]
        self.psnrs = list(st["psnrs"])
        self.last_reset, self.stop_iter, self.finetune_left = st["last_reset"], st["stop_iter"], st["finetune_left"]

    def thresholds(self, k: int) -> tuple[float, float]:
        c = self.cfg
        s = min(1.5, max(0.5, 0.5 + 1.5 * k / c.total_iter))
        return c.eps0_xyz * s, c.eps0_rgb * s

    def freeze_mode(self, k: int) -> int | None:
        """Freeze-map action before iteration k (None: nothing)."""
        c = self.cfg
        if not c.freezing or self.finetune_left is not None or k % c.every:
            return None
        end = c.window_end if self.stop_iter is None else min(c.window_end, self.stop_iter)
        if self.stop_iter is None and k == c.window_end:
            # freezing ends with the window: nothing stays frozen
            return FREEZE_RESET if c.window_end_reset else None
        if k >= end:
            return None
        if k < c.warmup:
            return FREEZE_CLEAR
        if k % c.reset_every == 0:
            self.last_reset = k
            return FREEZE_RESET
        if self.last_reset is not None and k - self.last_reset < c.wait:
            return FREEZE_CLEAR
        return FREEZE_CLEAR if c.freeze_strategy == "none" else FREEZE_UPDATE

    def lr_xyz_at(self, k: int) -> float:
        """xyz learning rate for iteration k: the plateau schedule under GSta,
        vanilla exponential decay for plain training."""
        c = self.cfg
        t = min(1.0, max(0.0, k / c.total_iter))
        if c.freezing:
            return self.lr_xyz * (c.plain_lr_final_ratio ** t if c.plateau_on_vanilla else 1.0)
        return self.lr_xyz * c.plain_lr_final_ratio ** t

    def wants_psnr(self, k: int) -> bool:
        c = self.cfg
        return c.freezing and self.finetune_left is None and k > 0 and k % c.psnr_every == 0 and k <= c.window_end

    def report_psnr(self, k: int, psnr: float) -> bool:
        """Record a subset PSNR; returns True when early stop fires (Eq. 7)."""
        c = self.cfg
        self.psnrs.append(psnr)
        if psnr > self._best + c.lr_eps:
            self._best, self._bad = psnr, 0
        else:
            self._bad += 1
            if self._bad > c.lr_patience:
                self.lr_xyz *= c.lr_decay
                self._bad = 0
        p = self.psnrs
        if len(p) >= 3 and p[-1] - p[-2] < c.eps_psnr and p[-2] - p[-3] < c.eps_psnr:
            self.stop_iter = k
            self.finetune_left = c.finetune_iters
            return True
        return False

    # ---- densification cadence ----
    def _den_end(self) -> int:
        c = self.cfg
        if not c.freezing:
            return c.den_until_plain
        return c.window_end if self.stop_iter is None else min(c.window_end, self.stop_iter)

    def densify_due(self, k: int) -> bool:
        """Densify and prune after iteration k: a multiple of den_every in (den_from, end)."""
        c = self.cfg
        return c.densify and self.finetune_left is None and k % c.den_every == 0 and c.den_from < k < self._den_end()

    def densify_uses_rgb(self, k: int) -> bool:
        return (k // self.cfg.den_every) % self.cfg.rgb_every == 0

    def opacity_reset_due(self, k: int) -> bool:
        c = self.cfg
        return (c.densify and self.finetune_left is None and k > 0 and k % c.opacity_every == 0
                and k <= self._den_end())

    def size_pruning(self, k: int) -> bool:
        return k > self.cfg.opacity_every

    def finished(self, k: int) -> bool:
        """Training ends after the finetuning stage (entered on early stop or at total_iter)."""
        if self.finetune_left is not None:
            return self.finetune_left <= 0
        return False

    def after_step(self, k: int) -> bool:
        """Advance the finetuning countdown; at total_iter without early stop, enter finetuning.
        Returns True when the map must be reset (all Gaussians unfrozen)."""
        c = self.cfg
        if self.finetune_left is not None:
            self.finetune_left -= 1
            return False
        if c.freezing and k + 1 >= c.total_iter:
            self.finetune_left = c.finetune_iters
            return True
        return False


def train_resolution(k: int, cfg: GStaConfig, W: int, H: int) -> tuple[int, int]:
    """Image size at iteration k under the progressive schedule: scale
    s = s0 + (1 - s0)(1 - cos(pi t)) / 2, t = min(k, K) / K, rounded per axis."""
    if not cfg.progressive:
        return W, H
    t = min(k, cfg.prog_until) / cfg.prog_until
    sc = cfg.prog_start + (1.0 - cfg.prog_start) * (1.0 - math.cos(math.pi * t)) / 2.0
    return max(1, int(round(sc * W))), max(1, int(round(sc * H)))


def blur_sigma(k: int, cfg: GStaConfig) -> float:
    """Blur standard deviation (pixels) at iteration k: sigma0 (1 + cos(pi t)) / 2."""
    if not cfg.blur:
        return 0.0
    t = min(k, cfg.blur_until) / cfg.blur_until
    return cfg.blur_sigma0 * (1.0 + math.cos(math.pi * t)) / 2.0


def mask_phase(k: int, cfg: GStaConfig) -> tuple[bool, bool]:
    """(masks applied, masks learned) at iteration k: applied from mask_from
    on, learned until mask_until."""
    if not cfg.volume_mask or k < cfg.mask_from:
        return False, False
    return True, k < cfg.mask_until


def mask_prune_due(k: int, cfg: GStaConfig) -> bool:
    """Prune masked-off Gaussians after iteration k: every mask_prune_every in [mask_from, mask_until]."""
    return (cfg.volume_mask and cfg.mask_from <= k <= cfg.mask_until and k > 0
            and k % cfg.mask_prune_every == 0)


def calibrate_eps0(cfg: GStaConfig, ctrl: GStaController, k: int, acc_xyz: np.ndarray, acc_rgb: np.ndarray,
                   cnt: np.ndarray):
    """Threshold calibration at the first freeze update (a reading, not in the
    paper: its initial thresholds were chosen by inspecting gradient magnitudes
    of real scenes, Sec. 4.1). If the configured thresholds at iteration k would
    freeze fewer than 5% or more than 95% of the visible Gaussians, returns
    ((eps0_xyz, eps0_rgb), frac) with initial values that put the threshold at
    iteration k on the 30th percentile of the averaged norms; else None."""
    vis = cnt > 0
    if vis.sum() == 0:
        return None
    ax = acc_xyz[vis] / cnt[vis]
    ar = acc_rgb[vis] / cnt[vis]
    ex, er = ctrl.thresholds(k)
    frac = float(np.mean((ax < ex) & (ar < er)))
    if 0.05 <= frac <= 0.95:
        return None
    scale = ex / cfg.eps0_xyz
    return (float(np.percentile(ax, 30)) / scale, float(np.percentile(ar, 30)) / scale), frac
