"""Device-resident state and the composition of one GSta training step.

Nothing here computes: it allocates the caller-owned buffers the C ABI
expects (PyTorch is the allocator) and calls the entry points in the order
of Algorithm 1 -- rasterise (project, sort, composite), loss, backward with
frozen Gaussians skipped, masked Adam -- plus the freeze-map update and the
PSNR check at the cadence the host controller decides.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import lib

# Learning rates per parameter group: xyz, scale, rotation, opacity, SH DC, SH rest.
# Sec. 4.1: the vanilla 3DGS rates except opacity 0.025; the vanilla values are
# not printed in the paper and are taken from common 3DGS practice: xyz
# 1.6e-4 x scene extent, scale 5e-3, rotation 1e-3, SH DC 2.5e-3, SH rest 2.5e-3/20.
def default_lrs(scene_extent: float) -> list[float]:
    return [1.6e-4 * scene_extent, 5e-3, 1e-3, 0.025, 2.5e-3, 2.5e-3 / 20.0]


def scaled_camera(cam: lib.GsCamera, W2: int, H2: int) -> lib.GsCamera:
    """The camera of a W2 x H2 image covering the same extent of the image
    plane (pixel j spans [j - 1/2, j + 1/2)): f' = f r, c' = (c + 1/2) r - 1/2."""
    c = lib.GsCamera.from_buffer_copy(cam)
    rx, ry = W2 / cam.width, H2 / cam.height
    c.width, c.height = int(W2), int(H2)
    c.fx, c.fy = cam.fx * rx, cam.fy * ry
    c.cx, c.cy = (cam.cx + 0.5) * rx - 0.5, (cam.cy + 0.5) * ry - 0.5
    return c


def pack_params(p59: np.ndarray, device="cuda") -> torch.Tensor:
    """(N, 59) array -> (N, 64) float32 device tensor with zero padding."""
    n = p59.shape[0]
    out = torch.zeros((n, lib.ROW), dtype=torch.float32)
    out[:, :59] = torch.from_numpy(np.ascontiguousarray(p59, dtype=np.float32))
    return out.to(device)


@dataclasses.dataclass
class View:
    """Per-resolution buffers of one rendered view."""
    cam: lib.GsCamera
    image: torch.Tensor
    t_final: torch.Tensor
    n_last: torch.Tensor
    dl: torch.Tensor
    loss: torch.Tensor
    loss_ws: torch.Tensor
    vals: torch.Tensor
    ranges: torch.Tensor
    count: torch.Tensor
    sort_ws: torch.Tensor
    capacity: int
    # the forward's record of where the backward resumes (trainable views;
    # gs_render_fwd_resume): [H W 4] float, [tiles] int32
    resume: torch.Tensor | None = None
    resume_pos: torch.Tensor | None = None


class Model:
    """Gaussian parameters, Adam moments, freeze state and per-step scratch on one GPU.

    Per-Gaussian buffers hold ``cap`` rows of which the first ``n`` are live;
    densification (``densify``) writes the new set into a spare copy of the
    parameters, moments and carried state, swaps, and grows every buffer
    (``generation`` counts the reallocations) when the set outgrows ``cap``."""

    def __init__(self, params59: np.ndarray, sh_degree: int = 3, device="cuda", trainable: bool = True,
                 capacity: int | None = None):
        self.device = torch.device(device)
        self.n = int(params59.shape[0])
        self.sh_degree = sh_degree
        self.trainable = trainable
        self.step_count = 0
        self.fwd_cfg = None  # rasteriser launch shapes (None: library defaults); see autotune.py
        self.bwd_cfg = None
        self.generation = 0
        self.den = None  # densification window statistics (enable_densify)
        self.opacity_act = lib.GS_OPACITY_SIGMOID  # GS_OPACITY_ABS after to_abs_opacity(), | GS_VOLUME_MASK
        self.mask_loss = 0.0  # lambda_m / N while the volume masks learn (set_volume_mask)
        self.mask_lr = None   # their learning rate (a seventh group), None: no mask
        self.carried: dict[str, torch.Tensor] = {}  # further per-Gaussian state moved by densify
        self._allocate(max(self.n, capacity or 0, 1))
        self.P[: self.n, :59] = torch.from_numpy(np.ascontiguousarray(params59, dtype=np.float32)).to(self.device)
        if trainable:
            self.act[: self.n] = torch.arange(self.n, dtype=torch.int32, device=self.device)
            self.n_active.fill_(self.n)

    def _allocate(self, cap: int):
        """Every per-Gaussian buffer at ``cap`` rows (zero)."""
        self.cap = cap
        f32 = dict(dtype=torch.float32, device=self.device)
        self.P = torch.zeros((cap, lib.ROW), **f32)
        self.splats = torch.zeros((cap, lib.SPLAT), **f32)
        if not self.trainable:  # render-only (targets): no gradients, moments or freeze state
            return
        self.G = torch.zeros((cap, lib.ROW), **f32)
        self.m = torch.zeros((cap, lib.ROW), **f32)
        self.v = torch.zeros((cap, lib.ROW), **f32)
        self.grad2d = torch.zeros((cap, lib.GRAD2D), **f32)
        self.frozen = torch.zeros(cap, dtype=torch.uint8, device=self.device)
        self.act = torch.zeros(cap, dtype=torch.int32, device=self.device)
        self.n_active = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.acc_xyz = torch.zeros(cap, **f32)
        self.acc_rgb = torch.zeros(cap, **f32)
        self.cnt = torch.zeros(cap, dtype=torch.int32, device=self.device)
        self.freeze_ws = torch.zeros(max(lib.gs_freeze_workspace_bytes(cap), 256), dtype=torch.uint8,
                                     device=self.device)
        self.select_ws = None  # gs_freeze_select workspace, made at first use
        if self.den is not None:
            self.enable_densify()

    # ---- densification (Sec. 4.1) ----
    def enable_densify(self):
        cap, f32 = self.cap, dict(dtype=torch.float32, device=self.device)
        self.den = dict(acc_xyz=torch.zeros(cap, **f32), acc_rgb=torch.zeros(cap, **f32),
                        cnt=torch.zeros(cap, dtype=torch.int32, device=self.device),
                        max_radius=torch.zeros(cap, dtype=torch.int32, device=self.device),
                        ws=torch.zeros(lib.gs_densify_workspace_bytes(cap), dtype=torch.uint8, device=self.device),
                        counts=torch.zeros(4, dtype=torch.int64, device=self.device))

    def carry(self, name: str, tensor: torch.Tensor):
        """Register a per-Gaussian tensor ([cap] or [cap][w]) that densification moves along."""
        self.carried[name] = tensor

    def _den_stats(self):
        d = self.den
        return lib.grad_stats(d["acc_xyz"], d["acc_rgb"], d["cnt"], d["max_radius"])

    def densify(self, prm: "lib.GsDensifyParams", rng: np.random.Generator) -> dict:
        """One densification and pruning step (gs_densify_plan / gs_densify_apply);
        returns the counts. Restarts the densification window; keeps the freeze
        window's statistics and the carried state of the surviving Gaussians."""
        if self.opacity_act & lib.GS_OPACITY_ABS:
            raise RuntimeError("densification thresholds are opacity logits: not under the absolute-value opacity")
        prune_only = self.den is None  # no candidates then: the freeze window stands in for the statistics
        if prune_only:
            if getattr(self, "_prune", None) is None or self._prune["ws"].numel() < lib.gs_densify_workspace_bytes(
                    self.cap):
                self._prune = dict(ws=torch.zeros(lib.gs_densify_workspace_bytes(self.cap), dtype=torch.uint8,
                                                  device=self.device),
                                   counts=torch.zeros(4, dtype=torch.int64, device=self.device))
            d, stats = self._prune, lib.grad_stats(self.acc_xyz, self.acc_rgb, self.cnt)
        else:
            d, stats = self.den, self._den_stats()
        n = self.n
        lib.gs_densify_plan(n, self.P, stats, prm, d["ws"], d["counts"])
        kept, clones, children, splits = (int(x) for x in d["counts"].cpu().tolist())
        n_out = kept + clones + children
        z = torch.from_numpy(rng.standard_normal((max(splits, 1), 2, 3)).astype(np.float32)).to(self.device)
        cap = self.cap if n_out <= self.cap else int(n_out * 1.5) + 1024
        f32 = dict(dtype=torch.float32, device=self.device)
        P2, m2, v2 = (torch.zeros((cap, lib.ROW), **f32) for _ in range(3))
        fr2 = torch.zeros(cap, dtype=torch.uint8, device=self.device)
        named = dict(acc_xyz=self.acc_xyz, acc_rgb=self.acc_rgb, cnt=self.cnt, **self.carried)
        out = {k: torch.zeros((cap,) + tuple(t.shape[1:]), dtype=t.dtype, device=self.device) for k, t in named.items()}
        carries = [lib.densify_carry(named[k], out[k]) for k in named]
        lib.gs_densify_apply(n, self.P, self.m, self.v, self.frozen, carries, prm, z, d["ws"], cap, P2, m2, v2, fr2)
        if cap != self.cap:  # grown: every other buffer anew
            if self.den is not None:
                self.den = dict(self.den)  # keep enable flag
            self._allocate(cap)
            self.generation += 1
        elif not prune_only:
            for key in ("acc_xyz", "acc_rgb", "cnt", "max_radius"):
                self.den[key].zero_()
        self.P, self.m, self.v, self.frozen = P2, m2, v2, fr2
        self.acc_xyz, self.acc_rgb, self.cnt = out["acc_xyz"], out["acc_rgb"], out["cnt"]
        for k in self.carried:
            self.carried[k] = out[k]
        self.n = n_out
        # the unfrozen list of the new set; map and freeze statistics kept
        lib.gs_freeze_update(self.n, self.acc_xyz, self.acc_rgb, self.cnt, self.frozen, 0.0, 0.0, 3, self.act,
                             self.n_active, self.freeze_ws)
        return dict(kept=kept, clones=clones, children=children, splits=splits, n=n_out)

    def prune_masked(self, logit_min: float, rng: np.random.Generator) -> dict:
        """Remove the Gaussians whose volume mask is off (Sec. 3.3): a
        densification pass with no candidates and only the mask rule."""
        inf = float("inf")
        prm = lib.GsDensifyParams(inf, inf, 0, 0.0, -inf, 0, 2**31 - 1, inf, 0.0, 1, logit_min)
        return self.densify(prm, rng)

    # ---- checkpoint ----
    _STATE = ("P", "G", "m", "v", "frozen", "act", "n_active", "acc_xyz", "acc_rgb", "cnt")

    def state_dict(self) -> dict:
        """Everything training needs to continue: parameters, gradients,
        moments, freeze map and list, both statistics windows, counters and
        the parameterisation (host copies)."""
        st = {k: getattr(self, k).detach().cpu().clone() for k in self._STATE}
        st.update(n=self.n, cap=self.cap, step_count=self.step_count, sh_degree=self.sh_degree,
                  opacity_act=self.opacity_act, mask_loss=self.mask_loss, mask_lr=self.mask_lr,
                  generation=self.generation)
        if self.den is not None:
            st["den"] = {k: t.detach().cpu().clone() for k, t in self.den.items()
                         if k in ("acc_xyz", "acc_rgb", "cnt", "max_radius")}
        return st

    def load_state_dict(self, st: dict):
        """Restore a state_dict (buffers reallocated at its capacity)."""
        self.sh_degree = st["sh_degree"]
        had_den = self.den is not None or "den" in st
        self.den = None
        self._allocate(st["cap"])
        for k in self._STATE:
            getattr(self, k).copy_(st[k].to(self.device))
        self.n, self.step_count = st["n"], st["step_count"]
        self.opacity_act, self.mask_loss, self.mask_lr = st["opacity_act"], st["mask_loss"], st["mask_lr"]
        self.generation = st["generation"] + 1  # buffers are new: views must be remade
        if had_den:
            self.enable_densify()
            for k, t in st.get("den", {}).items():
                self.den[k].copy_(t.to(self.device))
        self._step_key = None

    def prune_marked(self, mark: torch.Tensor, rng: np.random.Generator) -> dict:
        """Remove the Gaussians with mark[i] != 0 (uint8 [n], device): a
        densification pass with no candidates and only that rule."""
        inf = float("inf")
        prm = lib.GsDensifyParams(inf, inf, 0, 0.0, -inf, 0, 2**31 - 1, inf, 0.0, 0, 0.0,
                                  lib._ptr(mark, torch.uint8, "mark"))
        return self.densify(prm, rng)

    def significance_mark(self, hits: torch.Tensor, fraction: float, beta: float = 0.1,
                          quantile: float = 0.9) -> torch.Tensor:
        """Marks (uint8 [n]) of the floor(fraction n) least significant Gaussians
        given their hit counts over the training views (gs_significance_mark)."""
        mark = torch.zeros(max(self.n, 1), dtype=torch.uint8, device=self.device)
        ws = torch.zeros(lib.gs_significance_workspace_bytes(self.n), dtype=torch.uint8, device=self.device)
        lib.gs_significance_mark(self.n, self.P, hits, self.opacity_act, beta, quantile, fraction, mark, ws)
        return mark

    def set_volume_mask(self, on: bool, learn_lr: float | None = None, loss_weight: float = 0.0):
        """Volume masks (Sec. 3.3) applied (on) and, with learn_lr, learned with
        that rate and the mask term loss_weight * mean sigmoid(m)."""
        self.opacity_act = (self.opacity_act | lib.GS_VOLUME_MASK) if on else (
            self.opacity_act & ~lib.GS_VOLUME_MASK)
        self.mask_lr = learn_lr if on else None
        self.mask_loss = (loss_weight / max(self.n, 1)) if (on and learn_lr) else 0.0

    def opacity_reset(self, logit_cap: float, skip_frozen: bool = False):
        """Cap every opacity logit at logit_cap (moments zeroed), as 3DGS does;
        with skip_frozen the frozen Gaussians keep theirs."""
        if self.opacity_act & lib.GS_OPACITY_ABS:
            raise RuntimeError("the opacity reset caps a logit: not under the absolute-value opacity")
        lib.gs_opacity_reset(self.n, self.P, self.m, self.v, logit_cap, self.frozen if skip_frozen else None)

    # ---- views ----
    def make_view(self, cam: lib.GsCamera, capacity: int, trainable: bool = True) -> View:
        H, W = cam.height, cam.width
        dev = self.device
        return View(
            cam=cam,
            image=torch.zeros((3, H, W), dtype=torch.float32, device=dev),
            t_final=torch.zeros((H, W), dtype=torch.float32, device=dev),
            n_last=torch.zeros((H, W), dtype=torch.int32, device=dev),
            dl=torch.zeros((3, H, W) if trainable else (1,), dtype=torch.float32, device=dev),
            loss=torch.zeros(1, dtype=torch.float32, device=dev),
            loss_ws=torch.zeros(lib.gs_loss_workspace_bytes(H, W) if trainable else 1, dtype=torch.uint8,
                                device=dev),
            vals=torch.zeros(max(capacity, 1), dtype=torch.int32, device=dev),
            ranges=torch.zeros((cam.tiles, 2), dtype=torch.int32, device=dev),
            count=torch.zeros(1, dtype=torch.int64, device=dev),
            sort_ws=torch.zeros(lib.gs_sort_workspace_bytes(self.cap, capacity, cam), dtype=torch.uint8, device=dev),
            capacity=capacity,
            resume=torch.zeros(H * W * 4, dtype=torch.float32, device=dev) if trainable else None,
            resume_pos=torch.zeros(cam.tiles, dtype=torch.int32, device=dev) if trainable else None,
        )

    def retarget(self, view: View, cam: lib.GsCamera) -> View:
        """Same buffers, another camera with the same tile size and at most the
        resolution the buffers were made for (a smaller image uses a prefix)."""
        H0, W0 = view.image.shape[1], view.image.shape[2]
        assert cam.tile == view.cam.tile and cam.width * cam.height <= W0 * H0
        assert cam.width <= W0 and cam.height <= H0
        view.cam = cam
        return view

    # ---- step pieces ----
    def rasterize(self, view: View, stream=None):
        lib.gs_project_ex(self.P, self.n, self.sh_degree, self.opacity_act, view.cam, self.splats, stream)
        lib.gs_sort(self.splats, self.n, view.cam, view.sort_ws, view.capacity, view.vals, view.ranges, view.count,
                    stream)
        self.render_fwd(view, stream)

    def render_fwd(self, view: View, cfg=None, stream=None):
        """The compositing forward; on a trainable view it also records where
        the backward resumes (gs_render_fwd_resume)."""
        cfg = self.fwd_cfg if cfg is None else cfg
        if view.resume is not None:
            lib.gs_render_fwd_resume(self.splats, view.vals, view.ranges, view.cam, cfg, self.frozen, view.image,
                                     view.t_final, view.n_last, view.resume, view.resume_pos, stream)
        else:
            lib.gs_render_fwd_cfg(self.splats, view.vals, view.ranges, view.cam, cfg, view.image, view.t_final,
                                  view.n_last, stream)

    def raster_bwd(self, view: View, cfg=None, stream=None):
        """The rasteriser backward, from the forward's resume record when the
        view has one (the frozen splats behind a tile's last unfrozen one skipped)."""
        cfg = self.bwd_cfg if cfg is None else cfg
        if view.resume is not None:
            lib.gs_raster_bwd_resume(self.splats, view.vals, view.ranges, view.cam, cfg, view.t_final, view.n_last,
                                     view.dl, self.frozen, view.resume, view.resume_pos, self.grad2d, stream)
        else:
            lib.gs_raster_bwd_cfg(self.splats, view.vals, view.ranges, view.cam, cfg, view.t_final, view.n_last,
                                  view.dl, self.frozen, self.grad2d, stream)

    def loss(self, view: View, gt: torch.Tensor, lam: float = 0.2, stream=None):
        lib.gs_loss(view.image, gt, view.cam.height, view.cam.width, lam, view.loss_ws, view.loss, view.dl, stream)

    def backward(self, view: View, stats: bool = True, stream=None):
        """gs_render_bwd, as its two halves so that the tuned launch shape applies."""
        self.raster_bwd(view, stream=stream)
        self.project_backward(view, stats, stream)

    def project_backward(self, view: View, stats: bool = True, stream=None):
        """The projection half of the backward; it also feeds the densification
        window when that is enabled."""
        sets = []
        if stats:
            sets.append(lib.grad_stats(self.acc_xyz, self.acc_rgb, self.cnt))
            if self.den is not None:
                sets.append(self._den_stats())
        lib.gs_project_bwd_ex(self.P, self.n, self.sh_degree, self.opacity_act, view.cam, self.splats, self.act,
                              self.n_active, self.grad2d, self.G, False, sets, self.mask_loss, stream)

    def to_abs_opacity(self, moments: int = lib.GS_MOMENTS_ZERO, stream=None) -> float:
        """Switch to the absolute-value opacity of the finetuning stage (Sec. 4.1):
        gs_opacity_to_abs keeps every opacity; its Adam moments restart
        (GS_MOMENTS_ZERO) or are carried over (GS_MOMENTS_RESCALE). Returns
        the mean of sigmoid'(x) = o (1 - o) over the Gaussians at the switch."""
        if self.opacity_act & lib.GS_OPACITY_ABS:
            return 1.0
        acc = torch.zeros(1, dtype=torch.float32, device=self.device)
        lib.gs_opacity_to_abs(self.n, self.P, self.m, self.v, moments, acc, stream)
        self.opacity_act |= lib.GS_OPACITY_ABS
        return float(acc.item()) / max(self.n, 1)

    def apply_tuning(self, tuning):
        self.fwd_cfg = lib.raster_config(*tuning.fwd)
        self.bwd_cfg = lib.raster_config(*tuning.bwd)

    def adam(self, lrs, b1=0.9, b2=0.999, eps=1e-15, stream=None):
        self.step_count += 1
        lib.gs_adam_masked_groups(self.P, self.G, self.m, self.v, self.n, self.act, self.n_active,
                                  self._rates(lrs), b1, b2, eps, self.step_count, stream)

    def _rates(self, lrs) -> list:
        """The six group rates, and the volume masks' as a seventh while they learn."""
        return list(lrs) + ([self.mask_lr] if self.mask_lr else [])

    def train_step(self, view: View, gt: torch.Tensor, lrs, stream=None):
        """One iteration of Algorithm 1's inner body on the current freeze map:
        gs_train_step, the same kernels as rasterize / loss / backward / adam
        enqueued from native code in one call."""
        self.step_count += 1
        lib.gs_train_step(self._step_struct(view), view.cam, gt, self._rates(lrs), self.step_count, stream)

    def _step_struct(self, view: View) -> "lib.GsStep":
        """The gs_step of this model and view, rebuilt when a buffer or size changed."""
        den = self.den["acc_xyz"].data_ptr() if self.den is not None else 0
        key = (id(view), view.vals.data_ptr(), view.image.data_ptr(), view.capacity, self.P.data_ptr(),
               self.G.data_ptr(), self.m.data_ptr(), self.frozen.data_ptr(), self.acc_xyz.data_ptr(), den, self.n,
               self.opacity_act, self.mask_loss, bool(self.mask_lr), id(self.fwd_cfg), id(self.bwd_cfg))
        if getattr(self, "_step_key", None) != key:
            stats = [lib.grad_stats(self.acc_xyz, self.acc_rgb, self.cnt)]
            if self.den is not None:
                stats.append(self._den_stats())
            self._step = lib.step_args(self.P, self.G, self.m, self.v, self.splats, self.grad2d, self.n,
                                       self.sh_degree, self.opacity_act, self.frozen, self.act, self.n_active, stats,
                                       view.sort_ws, view.capacity, view.vals, view.ranges, view.count, view.image,
                                       view.t_final, view.n_last, view.dl, view.loss_ws, view.loss, 0.2, self.fwd_cfg,
                                       self.bwd_cfg, mask_loss=self.mask_loss, n_lr=7 if self.mask_lr else 6,
                                       resume=view.resume, resume_pos=view.resume_pos)
            self._step_key = key
        return self._step

    def freeze_select(self, eps_xyz: float, eps_rgb: float, strategy: int, fraction: float, u=None, stream=None):
        """A freeze update under one of the ablation strategies (lib.GS_FREEZE_*):
        gs_freeze_select; u: uniform draws [n] for the random strategy."""
        if self.select_ws is None:
            self.select_ws = torch.zeros(lib.gs_freeze_select_workspace_bytes(self.cap), dtype=torch.uint8,
                                         device=self.device)
        lib.gs_freeze_select(self.n, self.acc_xyz, self.acc_rgb, self.cnt, self.frozen, eps_xyz, eps_rgb, strategy,
                             fraction, u, self.act, self.n_active, self.select_ws, stream)

    def freeze_update(self, eps_xyz: float, eps_rgb: float, mode: int, stream=None):
        lib.gs_freeze_update(self.n, self.acc_xyz, self.acc_rgb, self.cnt, self.frozen, eps_xyz, eps_rgb, mode,
                             self.act, self.n_active, self.freeze_ws, stream)

    def measure_capacity(self, cams, slack: float = 1.25) -> int:
        """Largest entry count over ``cams`` (one projection + sort each), times ``slack``."""
        worst = 0
        for cam in cams:
            lib.gs_project_ex(self.P, self.n, self.sh_degree, self.opacity_act, cam, self.splats)
            tt = self.splats[:, 11].contiguous().view(torch.int32)
            worst = max(worst, int(tt.to(torch.int64).sum().item()))
        return int(worst * slack) + 1024


class TargetFeeder:
    """Targets from host memory for training from host buffers: each step's
    image is copied from pinned host memory into one of two device buffers
    on a copy stream, the copy of the next step's image overlapping the
    current step (the step waits for its own copy; a buffer is refilled only
    after the step that read it)."""

    def __init__(self, shape, device="cuda"):
        self.bufs = [torch.empty(shape, dtype=torch.float32, device=device) for _ in range(2)]
        self.copied = [torch.cuda.Event() for _ in range(2)]
        self.used = [torch.cuda.Event() for _ in range(2)]
        self.stream = torch.cuda.Stream(device=device)
        self.k = 0

    def prefetch(self, host: torch.Tensor):
        """Start copying the next step's target (pinned host tensor)."""
        b = self.k % 2
        with torch.cuda.stream(self.stream):
            self.stream.wait_event(self.used[b])  # the step that last read this buffer is done with it
            self.bufs[b].copy_(host, non_blocking=True)
            self.copied[b].record(self.stream)

    def take(self) -> torch.Tensor:
        """The buffer of the prefetched target, after the current stream waits for its copy."""
        b = self.k % 2
        torch.cuda.current_stream().wait_event(self.copied[b])
        return self.bufs[b]

    def release(self):
        """Mark the current buffer as read by the work enqueued so far; move on."""
        self.used[self.k % 2].record(torch.cuda.current_stream())
        self.k += 1
