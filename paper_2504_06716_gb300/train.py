"""GSta training loop (Algorithm 1) on one GPU over the C ABI.

Per iteration: freeze-map action at the schedule's cadence (Eqs. 4-6),
subset PSNR and early-stop check every 1000 iterations (Eq. 7), then
rasterise, loss, backward with frozen Gaussians skipped and masked Adam on
the sampled training view. Targets are rendered once from the ground-truth
Gaussian set with the same CUDA renderer.

Threshold calibration (a reading, not in the paper): the paper chose its
initial thresholds by looking at gradient magnitudes of real scenes
(Sec. 4.1). If, at the first update, those values would freeze fewer than 5%
or more than 95% of the visible Gaussians of a synthetic scene, the initial
thresholds are re-chosen so that the threshold at that iteration equals the
30th percentile of the observed averaged norms.

Run as a script for a full training run:
  python -m paper_2504_06716_gb300.train --arm gsta|plain [--n-init ...]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import autotune, lib, pipeline, synth
from .schedule import (FREEZE_RESET, FREEZE_UPDATE, GStaConfig, GStaController, blur_sigma, calibrate_eps0,
                       mask_phase, mask_prune_due, train_resolution)


class JsonlLog:
    """Training record as JSON lines, one object per line.

    Every ``every`` iterations: ``{"k", "loss", "n", "n_active",
    "frozen_frac", "entries", "lr_xyz"}`` for the step just taken (k is that
    step's iteration; loss is its training loss; entries the (Gaussian, tile)
    pairs its sort produced). Schedule events (subset PSNR checks, early stop,
    densification, prunes, resets) are written as ``{"k", "event", "value"}``
    when they have happened, and held-out evaluations as ``{"k", "eval", ...}``.
    Reading the loss and the counts waits for the step, so the cadence sets
    what the log costs."""

    def __init__(self, path: str, every: int = 100):
        if every < 1:
            raise ValueError("every must be >= 1")
        self.f = open(path, "w")
        self.every = every
        self._events_seen = 0

    def _write(self, rec: dict):
        self.f.write(json.dumps(rec) + "\n")

    def after_iteration(self, tr):
        for k, kind, value in tr.events[self._events_seen:]:
            self._write(dict(k=int(k), event=kind, value=float(value)))
        self._events_seen = len(tr.events)
        k = tr.k - 1
        if k < 0 or k % self.every:
            return
        m = tr.model
        n, n_active = int(m.n), int(m.n_active.item())
        self._write(dict(k=k, loss=float(tr.view.loss.item()), n=n, n_active=n_active,
                         frozen_frac=(n - n_active) / n if n else 0.0, entries=int(tr.view.count.item()),
                         lr_xyz=float(tr.ctrl.lr_xyz_at(k))))

    def evaluation(self, rec: dict):
        self._write(dict(k=int(rec["k"]), eval=True, **{a: b for a, b in rec.items() if a != "k"}))

    def close(self):
        self.f.close()


class Trainer:
    def __init__(self, scene: synth.Scene, cfg: GStaConfig, tile: int = 16, calibrate: bool = True,
                 extent: float = 4.4, seed: int = 3, device="cuda", target_noise: float = 0.0):
        self.scene = scene
        self.cfg = cfg
        self.calibrate = calibrate
        self.cams = [lib.camera(c, tile=tile) for c in scene.cameras]
        self.device = torch.device(device)
        # targets rendered from the ground-truth set
        gt_views = sorted(set(scene.train_views) | set(scene.test_views))
        gtm = pipeline.Model(scene.gt, device=self.device, trainable=False)
        gcap = gtm.measure_capacity([self.cams[v] for v in gt_views])
        gv = gtm.make_view(self.cams[gt_views[0]], gcap, trainable=False)
        self.targets = {}
        for v in gt_views:
            gtm.retarget(gv, self.cams[v])
            gtm.rasterize(gv)
            self.targets[v] = gv.image.clone()
            if target_noise > 0:  # sensor noise of a captured image, drawn per view on the host
                g = torch.Generator().manual_seed(7919 * (v + 1))
                noise = torch.randn(gv.image.shape, generator=g) * target_noise
                self.targets[v] = (self.targets[v] + noise.to(self.device)).clamp_(0.0, 1.0)
        if lib.gs_get_device_error():
            raise RuntimeError("device error while rendering targets")
        del gtm, gv
        self.extent = extent
        self.seed = seed
        self.fresh_model()
        H, W = self.cams[0].height, self.cams[0].width
        self.psnr_ws = torch.zeros(lib.gs_psnr_workspace_bytes(1, H, W), dtype=torch.uint8, device=self.device)
        # targets of the progressive / blur schedules (prefixes used at the reduced size)
        self.sched_buf = [torch.zeros(3 * H * W, dtype=torch.float32, device=self.device) for _ in range(2)]
        self.psnr_out = torch.zeros(1, device=self.device)
        self.lrs = pipeline.default_lrs(extent)
        if not cfg.freezing:  # plain 3DGS: vanilla opacity rate
            self.lrs[3] = cfg.plain_opacity_lr
        self.ctrl = GStaController(cfg, self.lrs[0])
        self.order = synth.view_order(cfg.total_iter + cfg.finetune_iters + 1, scene.train_views, seed)
        self.eps0 = (cfg.eps0_xyz, cfg.eps0_rgb)
        self.calibrated = False
        self.events: list[tuple[int, str, float]] = []
        self.k = 0
        self.active_iters = 0  # sum over iterations of the unfrozen count (the work freezing saves)
        self._act_now = None   # that count, re-read after each change of the freeze map or set
        self.capacity_check_every = 100
        self.overflows = 0
        # learned freeze predictor (predictor.py): state, logging, application
        self.pred_state = None
        self.log = None
        self.predictor = None
        self.pred_tau, self.pred_every = 0.9, 100
        self.pred_count = 0
        self.shadow = False  # evaluation: judge newly frozen Gaussians on their unmasked gradients
        self.shadow_checked = {"rule": 0, "pred": 0}
        self.shadow_false = {"rule": 0, "pred": 0}
        self._shadow_sets = {}

    def fresh_model(self, tuning=None):
        """The trainable model at its initialisation (and its view buffers)."""
        scene, cfg = self.scene, self.cfg
        self.model = pipeline.Model(scene.init, device=self.device,
                                    capacity=int(scene.init.shape[0] * (1.5 if cfg.densify else 1.0)))
        if cfg.densify:
            self.model.enable_densify()
        if cfg.volume_mask:  # every Gaussian starts with its mask on
            self.model.P[: self.model.n, 59] = cfg.mask_init
        if tuning is not None:
            self.model.apply_tuning(tuning)
        self.den_rng = np.random.default_rng(self.seed + 1000)  # the split draws
        self.freeze_rng = np.random.default_rng(self.seed + 2000)  # draws of the random freeze strategy
        vis = sorted(set(scene.train_views) | set(scene.test_views))
        cap = self.model.measure_capacity([self.cams[v] for v in vis])
        self.view = self.model.make_view(self.cams[scene.train_views[0]], cap)
        self.generation = self.model.generation

    def enable_predictor_state(self):
        if self.cfg.densify:
            raise NotImplementedError("the learned predictor is evaluated without densification")
        n, dev = self.model.n, self.device
        self.pred_state = torch.zeros((n, 12), dtype=torch.float32, device=dev)
        self.pred_X = torch.zeros((n, 16), dtype=torch.bfloat16, device=dev)
        self.pred_p = torch.zeros(n, dtype=torch.float32, device=dev)

    def _features(self, k: int, ex: float, er: float):
        m = self.model
        lib.gs_pred_features(m.n, m.P, m.acc_xyz, m.acc_rgb, m.cnt, self.pred_state, k, self.cfg.total_iter, ex, er,
                             self.pred_X)
        return self.pred_X

    def _predictor_due(self, k: int) -> bool:
        c, cfg = self.ctrl, self.cfg
        if self.predictor is None or not cfg.freezing or c.finetune_left is not None or k % self.pred_every:
            return False
        end = cfg.window_end if c.stop_iter is None else min(cfg.window_end, c.stop_iter)
        if k < cfg.warmup or k >= end:
            return False
        return c.last_reset is None or k - c.last_reset >= cfg.wait

    def _apply_predictor(self, k: int):
        m = self.model
        ex, er = self.thresholds(k)
        X = self._features(k, ex, er)
        self.predictor.predict(X, self.pred_p)
        before = m.frozen.clone() if self.shadow else None
        n0 = int(m.n_active.item())
        lib.gs_freeze_apply(m.n, self.pred_p, self.pred_tau, m.frozen, m.act, m.n_active, m.freeze_ws)
        self.pred_count += n0 - int(m.n_active.item())
        if self.shadow:
            self._track("pred", (m.frozen == 1) & (before == 0))

    def _track(self, source: str, newly):
        cur = self._shadow_sets.get(source)
        self._shadow_sets[source] = newly if cur is None else (cur | newly)

    def _shadow_backward(self):
        """Evaluation only: the unmasked gradient statistics of the Gaussians the
        predictor froze in this window (no update is applied)."""
        m, v = self.model, self.view
        if not hasattr(self, "_sh"):
            n = m.n
            self._sh = dict(g2d=torch.zeros_like(m.grad2d), G=torch.zeros_like(m.G),
                            ax=torch.zeros(n, device=self.device), ar=torch.zeros(n, device=self.device),
                            cnt=torch.zeros(n, dtype=torch.int32, device=self.device))
        sh = self._sh
        union = None
        for mask in self._shadow_sets.values():
            union = mask if union is None else (union | mask)
        idx = torch.nonzero(union).flatten().to(torch.int32)
        if idx.numel() == 0:
            return
        sh["g2d"].zero_()
        lib.gs_raster_bwd_cfg(m.splats, v.vals, v.ranges, v.cam, m.bwd_cfg, v.t_final, v.n_last, v.dl, None,
                              sh["g2d"])
        lib.gs_project_bwd(m.P, m.n, m.sh_degree, v.cam, m.splats, idx,
                           torch.tensor([idx.numel()], dtype=torch.int32, device=self.device), sh["g2d"], sh["G"],
                           sh["ax"], sh["ar"], sh["cnt"])

    def _close_shadow_window(self, ex: float, er: float):
        """At a statistics boundary: a Gaussian frozen during the window just ended
        counts as a false freeze if its unmasked averages over that window would
        not have passed the rule (Eq. 4/6)."""
        if self._shadow_sets and hasattr(self, "_sh"):
            sh = self._sh
            c = sh["cnt"].clamp(min=1).float()
            over = (sh["ax"] / c >= ex) | (sh["ar"] / c >= er)
            for src, mask in self._shadow_sets.items():
                seen = mask & (sh["cnt"] > 0)
                self.shadow_checked[src] += int(seen.sum().item())
                self.shadow_false[src] += int((seen & over).sum().item())
            sh["ax"].zero_()
            sh["ar"].zero_()
            sh["cnt"].zero_()
        self._shadow_sets = {}

    def false_freeze_rate(self, source: str = "pred") -> float | None:
        n = self.shadow_checked[source]
        return self.shadow_false[source] / n if n else None

    def check_capacity(self, headroom: float = 0.8, grow: float = 1.5):
        """Read the sort's entry count and the device error word (one sync) and
        grow the sort buffers before the count reaches the capacity. An
        overflow that already happened (truncated lists) is counted."""
        P = int(self.view.count.item())
        flags = lib.gs_get_device_error()
        if flags & lib.GS_FLAG_CAPACITY:
            self.overflows += 1
            self.events.append((self.k, "capacity_overflow", float(P)))
        if flags & ~lib.GS_FLAG_CAPACITY:
            raise RuntimeError(f"device error flags {flags:#x} at iteration {self.k}")
        if P > headroom * self.view.capacity:
            cam = self.view.cam
            self.view = self.model.make_view(cam, int(max(P, self.view.capacity) * grow) + 1024)
            self.events.append((self.k, "capacity", float(self.view.capacity)))

    def autotune(self, n_views: int = 2) -> autotune.RasterTuning:
        """Pick the rasteriser tile size and launch shapes on the current state
        (autotune.py) and switch every camera and buffer to them."""
        views = [self.order[(self.k + i) % len(self.order)] for i in range(n_views)]
        res = autotune.tune(self.model, [self.cams[v] for v in views], [self.targets[v] for v in views],
                            n_views=n_views)
        self.cams = [autotune.retile(c, res.tile) for c in self.cams]
        vis = sorted(set(self.scene.train_views) | set(self.scene.test_views))
        cap = self.model.measure_capacity([self.cams[v] for v in vis])
        self.view = self.model.make_view(self.cams[self.scene.train_views[0]], cap)
        self.model.apply_tuning(res)
        self.tuning = res
        return res

    # ---- measurements ----
    def psnr_of(self, views) -> float:
        vals = []
        for v in views:
            self.model.retarget(self.view, self.cams[v])
            self.model.rasterize(self.view)
            lib.gs_psnr(self.view.image, self.targets[v], 1, self.view.cam.height, self.view.cam.width, self.psnr_ws,
                        self.psnr_out)
            vals.append(self.psnr_out.clone())
        return float(torch.stack(vals).mean().item())

    def heldout_psnr(self) -> float:
        return self.psnr_of(self.scene.test_views)

    # ---- thresholds ----
    def _maybe_calibrate(self, k: int):
        if self.calibrated or not self.calibrate:
            return
        self.calibrated = True
        m = self.model
        res = calibrate_eps0(self.cfg, self.ctrl, k, m.acc_xyz.cpu().numpy(), m.acc_rgb.cpu().numpy(),
                             m.cnt.cpu().numpy())
        if res is not None:
            self.eps0 = res[0]
            self.events.append((k, "calibrated", res[1]))

    def thresholds(self, k: int) -> tuple[float, float]:
        ex, er = self.ctrl.thresholds(k)
        return ex * self.eps0[0] / self.cfg.eps0_xyz, er * self.eps0[1] / self.cfg.eps0_rgb

    # ---- one iteration of Algorithm 1 ----
    def iteration(self, allow_early_stop: bool = True):
        k = self.k
        m, c = self.model, self.ctrl
        mode = c.freeze_mode(k)
        if mode is not None or self._predictor_due(k):
            self._act_now = None
        if mode is not None:
            if mode == FREEZE_UPDATE:
                self._maybe_calibrate(k)
            ex, er = self.thresholds(k)
            if self.pred_state is not None:
                if self.log is not None and mode == FREEZE_UPDATE:
                    self.log.features.append((k, self._features(k, ex, er).clone()))
                if self.shadow:
                    self._close_shadow_window(ex, er)
                lib.gs_pred_history(m.n, m.acc_xyz, m.acc_rgb, m.cnt, m.frozen, self.pred_state)
            before = m.frozen.clone() if (self.shadow and mode == FREEZE_UPDATE) else None
            self._freeze(ex, er, mode)
            if before is not None:
                self._track("rule", (m.frozen == 1) & (before == 0))
            if self.log is not None:
                if mode == FREEZE_UPDATE:
                    self.log.frozen_after.append((k, m.frozen.cpu().numpy()))
                elif mode == FREEZE_RESET:
                    self.log.resets.append(k)
        elif self._predictor_due(k):
            self._apply_predictor(k)
        if c.wants_psnr(k):
            p = self.psnr_of(self.scene.subset_views)
            stop = c.report_psnr(k, p)
            self.events.append((k, "psnr", p))
            if stop and allow_early_stop:
                m.freeze_update(0.0, 0.0, FREEZE_RESET)
                self._act_now = None
                self._enter_finetune()
                self.events.append((k, "early_stop", p))
            elif stop:
                c.stop_iter, c.finetune_left = None, None
        v = self.order[k]
        cam, gt = self._scheduled_view(k, v)
        m.retarget(self.view, cam)
        lrs = list(self.lrs)
        lrs[0] = c.lr_xyz_at(k)
        if self._act_now is None:
            self._act_now = int(m.n_active.item())
        self.active_iters += self._act_now
        if self.cfg.volume_mask:
            applied, learned = mask_phase(k, self.cfg)
            m.set_volume_mask(applied, self.cfg.mask_lr if learned else None, self.cfg.mask_lambda)
        m.train_step(self.view, gt, lrs)
        if self.shadow and self._shadow_sets:
            self._shadow_backward()
        if c.densify_due(k):
            self._densify(k)
            self._act_now = None
        if self.cfg.significance and k in self.cfg.sig_iters and c.finetune_left is None:
            self._significance_prune(k)
        if mask_prune_due(k, self.cfg) and c.finetune_left is None:
            res = m.prune_masked(float(np.float32(math.log(0.01 / 0.99))), self.den_rng)
            self.events.append((k, "mask_prune", float(res["n"])))
            self._act_now = None
            if m.generation != self.generation:
                self.generation = m.generation
                self.view = m.make_view(self.view.cam, self.view.capacity)
        if c.opacity_reset_due(k):
            how = self.cfg.opacity_reset_frozen
            m.opacity_reset(float(np.float32(math.log(0.01 / 0.99))), skip_frozen=(how == "skip"))
            if how == "unfreeze" and self.cfg.freezing:
                m.freeze_update(0.0, 0.0, FREEZE_RESET)
                self._act_now = None
            self.events.append((k, "opacity_reset", 0.0))
        if c.after_step(k):
            m.freeze_update(0.0, 0.0, FREEZE_RESET)
            self._act_now = None
            self._enter_finetune()
        self.k += 1
        if self.k % self.capacity_check_every == 0:
            self.check_capacity()

    def _significance_prune(self, k: int):
        """Significance pruning (Sec. 3.3): hit counts over every training view
        (gs_hit_counts after each view's forward), scores, marks, removal."""
        m = self.model
        hits = torch.zeros(max(m.n, 1), dtype=torch.int32, device=self.device)
        for v in self.scene.train_views:
            m.retarget(self.view, self.cams[v])
            m.rasterize(self.view)
            lib.gs_hit_counts(m.splats, self.view.vals, self.view.ranges, self.view.cam, self.view.n_last, hits)
        i = list(self.cfg.sig_iters).index(k)
        frac = self.cfg.sig_fraction * self.cfg.sig_decay ** i
        mark = m.significance_mark(hits, frac, self.cfg.sig_beta, self.cfg.sig_quantile)
        res = m.prune_marked(mark, self.den_rng)
        self.events.append((k, "significance_prune", float(res["n"])))
        self._act_now = None
        if m.generation != self.generation:
            self.generation = m.generation
            self.view = m.make_view(self.view.cam, self.view.capacity)

    # ---- checkpoint / resume ----
    def save_checkpoint(self, path: str):
        """Model, controller and trainer state (iteration, thresholds, lrs,
        random generators, events) in one file: resuming continues the run."""
        torch.save(dict(model=self.model.state_dict(), ctrl=self.ctrl.state_dict(), k=self.k, eps0=self.eps0,
                        calibrated=self.calibrated, lrs=list(self.lrs), events=list(self.events),
                        active_iters=self.active_iters, overflows=self.overflows,
                        den_rng=self.den_rng.bit_generator.state, freeze_rng=self.freeze_rng.bit_generator.state,
                        capacity=self.view.capacity), path)

    def load_checkpoint(self, path: str):
        st = torch.load(path, weights_only=False)
        self.model.load_state_dict(st["model"])
        self.ctrl.load_state_dict(st["ctrl"])
        self.k, self.eps0, self.calibrated = st["k"], tuple(st["eps0"]), st["calibrated"]
        self.lrs, self.events, self.active_iters = list(st["lrs"]), list(st["events"]), st["active_iters"]
        self.overflows = st["overflows"]
        self.den_rng.bit_generator.state = st["den_rng"]
        self.freeze_rng.bit_generator.state = st["freeze_rng"]
        self._act_now = None
        self.generation = self.model.generation
        self.view = self.model.make_view(self.view.cam, st["capacity"])
        if getattr(self, "tuning", None) is not None:
            self.model.apply_tuning(self.tuning)

    def _scheduled_view(self, k: int, v: int):
        """Camera and target of view v at iteration k: the full-resolution ones,
        or under the progressive / blur schedules (Sec. 3.3) the area-averaged
        target at the scheduled size (gs_resize_area), blurred (gs_blur)."""
        cam, gt = self.cams[v], self.targets[v]
        W, H = cam.width, cam.height
        W2, H2 = train_resolution(k, self.cfg, W, H)
        sigma = float(np.float32(blur_sigma(k, self.cfg)))
        if (W2, H2) == (W, H) and sigma < lib.GS_BLUR_SIGMA_MIN:
            return cam, gt
        a, b = (t[: 3 * H2 * W2].view(3, H2, W2) for t in self.sched_buf)
        if (W2, H2) != (W, H):
            lib.gs_resize_area(gt, 3, W, H, a, W2, H2)
            cam, gt = pipeline.scaled_camera(cam, W2, H2), a
        if sigma >= lib.GS_BLUR_SIGMA_MIN:
            lib.gs_blur(gt, 3, W2, H2, sigma, b)
            gt = b
        return cam, gt

    def _enter_finetune(self):
        """Start of the finetuning stage: all Gaussians unfrozen (done by the
        caller) and, as in Sec. 4.1, the absolute-value opacity."""
        if self.cfg.abs_opacity_finetune:
            slope = self.model.to_abs_opacity(lib.GS_MOMENTS_RESCALE if self.cfg.abs_opacity_moments == "rescale"
                                              else lib.GS_MOMENTS_ZERO)
            self.lrs = list(self.lrs)
            if self.cfg.abs_opacity_lr == "slope":  # keep the mean opacity step of an Adam update
                self.lrs[3] *= slope
            elif self.cfg.abs_opacity_lr is not None:
                self.lrs[3] = float(self.cfg.abs_opacity_lr)
            self.events.append((self.k, "abs_opacity", self.lrs[3]))

    STRATEGIES = {"gsta": lib.GS_FREEZE_RULE, "xyz": lib.GS_FREEZE_XYZ, "random": lib.GS_FREEZE_RANDOM,
                  "mingrad": lib.GS_FREEZE_MINGRAD}

    def _freeze(self, ex: float, er: float, mode: int):
        """The freeze-map action: Eq. 4 (gs_freeze_update) or, for an update
        under an ablation strategy, gs_freeze_select."""
        m, strategy = self.model, self.cfg.freeze_strategy
        if mode != FREEZE_UPDATE or strategy == "gsta":
            m.freeze_update(ex, er, mode)
            return
        u = None
        if strategy == "random":
            u = torch.from_numpy(self.freeze_rng.random(max(m.n, 1), dtype=np.float32)).to(self.device)
        m.freeze_select(ex, er, self.STRATEGIES[strategy], self.cfg.freeze_fraction, u)

    # ---- densification (Sec. 4.1) ----
    def densify_params(self, k: int) -> lib.GsDensifyParams:
        cfg, c = self.cfg, self.ctrl
        s = min(1.5, max(0.5, 0.5 + 1.5 * k / cfg.total_iter))  # dynamic thresholds, as Eq. 5
        f = lambda x: float(np.float32(x))  # noqa: E731
        return lib.GsDensifyParams(f(cfg.eps0_den_xyz * s), f(cfg.eps0_den_rgb * s), int(c.densify_uses_rgb(k)),
                                   f(math.log(cfg.percent_dense * self.extent)),
                                   f(math.log(cfg.min_opacity / (1 - cfg.min_opacity))), int(c.size_pruning(k)),
                                   2**31 - 1 if cfg.max_screen_radius is None else cfg.max_screen_radius,
                                   f(math.log(cfg.max_world_frac * self.extent)),
                                   f(math.log(cfg.split_div)))

    def _densify(self, k: int):
        m = self.model
        res = m.densify(self.densify_params(k), self.den_rng)
        self.events.append((k, "densify", float(res["n"])))
        if m.generation != self.generation:  # buffers grew: views anew
            self.generation = m.generation
            self.view = m.make_view(self.view.cam, self.view.capacity)

    def finished(self) -> bool:
        c = self.ctrl
        if c.finetune_left is not None:
            return c.finetune_left <= 0
        return self.k >= self.cfg.total_iter and not self.cfg.freezing


def run(args, scene: synth.Scene | None = None) -> dict:
    """One training run as the arguments of parser() say, on the current CUDA
    device; the surface scene is generated unless one is given."""
    if scene is None:
        scene = synth.surface_scene(args.n_init, args.n_gt, args.views, args.width, args.height)
    cfg = GStaConfig(freezing=(args.arm == "gsta"), total_iter=args.iters, densify=not args.no_densify,
                     freeze_strategy=args.freeze_strategy, abs_opacity_finetune=not args.no_abs_opacity,
                     abs_opacity_moments=args.abs_moments,
                     abs_opacity_lr=None if args.abs_lr == "same" else
                     ("slope" if args.abs_lr == "slope" else float(args.abs_lr)),
                     progressive=args.trick_gs, blur=args.trick_gs, volume_mask=args.trick_gs or args.volume_mask,
                     significance=args.trick_gs or args.significance, early_stop=not args.no_early_stop,
                     window_end_reset=not args.no_window_end_reset, opacity_reset_frozen=args.opacity_reset_frozen,
                     eps0_xyz=3e-5 * args.eps_scale, eps0_rgb=1e-4 * args.eps_scale,
                     plateau_on_vanilla=not args.plateau_alone)
    tr = Trainer(scene, cfg, calibrate=not args.no_calibrate, target_noise=args.target_noise)
    tuning = None
    if args.autotune:
        for _ in range(args.tune_after):
            tr.iteration()
        tuning = dict(tile=tr.autotune().tile, fwd=tr.tuning.fwd, bwd=tr.tuning.bwd)
        tr2 = Trainer.__new__(Trainer)  # restart training from the initial state with the tuned shapes
        tr2.__dict__.update(tr.__dict__)
        tr2.fresh_model(tr.tuning)
        tr2.ctrl = GStaController(cfg, tr.lrs[0])
        tr2.k, tr2.calibrated, tr2.eps0, tr2.events, tr2.overflows = 0, False, (cfg.eps0_xyz, cfg.eps0_rgb), [], 0
        tr2.active_iters, tr2._act_now = 0, None
        tr = tr2
    evals = []
    log = JsonlLog(args.log_jsonl, args.log_every) if getattr(args, "log_jsonl", None) else None
    t0 = time.perf_counter()
    eval_every = args.eval_every
    while not tr.finished():
        tr.iteration(allow_early_stop=cfg.early_stop)
        if log is not None:  # counted as training time (a short wait every log.every iterations)
            log.after_iteration(tr)
        if tr.k % eval_every == 0:
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            evals.append(dict(k=tr.k, wall_s=el, heldout_psnr=tr.heldout_psnr(), n=tr.model.n,
                              n_active=int(tr.model.n_active.item())))
            if log is not None:
                log.evaluation(evals[-1])
            t0 = time.perf_counter() - el  # held-out evaluation is not training time
    torch.cuda.synchronize()
    total = time.perf_counter() - t0
    if log is not None:
        log.close()
    out = dict(arm=args.arm, freeze_strategy=cfg.freeze_strategy, abs_opacity_finetune=cfg.abs_opacity_finetune,
               trick_gs=args.trick_gs,
               abs_opacity_moments=cfg.abs_opacity_moments,
               calibrate=not args.no_calibrate, iters=tr.k, train_s=total, final_heldout_psnr=tr.heldout_psnr(),
               active_gaussian_iters=tr.active_iters, evals=evals,
               events=[e for e in tr.events if e[1] != "densify"], n_final=tr.model.n,
               densify=[e for e in tr.events if e[1] == "densify"][::10], eps0=tr.eps0, tuning=tuning, overflows=tr.overflows,
               final_capacity=tr.view.capacity, device_flags=lib.gs_get_device_error())
    return out


def parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument("--arm", choices=["gsta", "plain"], default="gsta")
    ap.add_argument("--n-init", type=int, default=1_000_000)
    ap.add_argument("--n-gt", type=int, default=1_500_000)
    ap.add_argument("--views", type=int, default=200)
    ap.add_argument("--width", type=int, default=1237)
    ap.add_argument("--height", type=int, default=822)
    ap.add_argument("--iters", type=int, default=30000)
    ap.add_argument("--eval-every", type=int, default=1000)
    ap.add_argument("--autotune", action="store_true", help="tune the rasteriser launch shape first")
    ap.add_argument("--no-calibrate", action="store_true", help="use the paper's initial thresholds as they are")
    ap.add_argument("--no-densify", action="store_true", help="keep the Gaussian set fixed")
    ap.add_argument("--tune-after", type=int, default=300, help="iterations trained before tuning (then restarted)")
    ap.add_argument("--freeze-strategy", choices=["gsta", "xyz", "random", "mingrad", "none"], default="gsta",
                    help="freeze rule or an ablation variant (Sec. 5, Table 3)")
    ap.add_argument("--no-abs-opacity", action="store_true",
                    help="keep the sigmoid opacity activation in the finetuning stage")
    ap.add_argument("--abs-moments", choices=["zero", "rescale"], default="rescale",
                    help="the opacity's Adam moments when the finetuning stage switches to |x|")
    ap.add_argument("--trick-gs", action="store_true",
                    help="progressive resolution and blur of the targets until 6K, volume masks, significance"
                         " pruning (Sec. 3.3)")
    ap.add_argument("--volume-mask", action="store_true", help="volume masks only (Sec. 3.3)")
    ap.add_argument("--significance", action="store_true", help="significance pruning only (Sec. 3.3)")
    ap.add_argument("--abs-lr", default="slope",
                    help="opacity learning rate under |x|: 'slope' (the rate times the mean o (1 - o) at the"
                         " switch), 'same' (unchanged) or a number")
    ap.add_argument("--no-early-stop", action="store_true", help="Eq. 7 never ends the run (PSNR still checked)")
    ap.add_argument("--no-window-end-reset", action="store_true",
                    help="keep the map when the freezing window closes without an early stop")
    ap.add_argument("--opacity-reset-frozen", choices=["reset", "skip", "unfreeze"], default="skip",
                    help="the opacity reset on frozen Gaussians: leave them, cap them too, or cap all and reset the map")
    ap.add_argument("--plateau-alone", action="store_true",
                    help="the plateau decays replace the vanilla exponential xyz schedule (a constant rate between "
                         "decays) instead of multiplying it")
    ap.add_argument("--target-noise", type=float, default=0.0,
                    help="standard deviation of seeded per-pixel noise added to every target image")
    ap.add_argument("--eps-scale", type=float, default=1.0, help="factor on the paper's initial freeze thresholds")
    ap.add_argument("--log-jsonl", default=None, help="write a per-iteration training record (JSON lines) here")
    ap.add_argument("--log-every", type=int, default=100, help="iterations between records of --log-jsonl")
    return ap


def main():
    torch.cuda.set_device(0)
    print(json.dumps(run(parser().parse_args())))


if __name__ == "__main__":
    main()
