"""Several scenes of uneven size trained together, one step for all of them.

The workload: 8 scenes of 50K, 120K, 250K, 400K, 600K, 900K, 1.4M and 2M
Gaussians (SH degree 3, float32) rendered at 800x800, each scene taking an
optimiser step over 4 of its training views per batch step, with GSta
freezing on (Sec. 3.2). One batch step:

  per (scene, view)  gs_project, gs_sort into the slot's own buffers
  all jobs           gs_render_fwd_batch: ONE persistent launch over the
                     8 x 4 (scene, view) jobs; CTAs take (job, tile) items
                     from a device counter, so a 2M-Gaussian view and a
                     50K-Gaussian view share the GPU without a launch each
  per (scene, view)  gs_loss (Eq. 3)
  all jobs           gs_raster_bwd_batch: ONE persistent launch, frozen
                     Gaussians skipped (Sec. 3.2.4)
  per scene          gs_project_bwd for its first view, gs_project_bwd_accum
                     for the others (the scene's gradient is the sum over its
                     4 views; the freeze statistics count each view), then
                     gs_adam_masked_devstep over the scene's active list

The training views of a scene are split into fixed groups of 4; the batch
step for group g is captured once into a CUDA graph and replayed. Nothing a
graph bakes in changes between replays: cameras, buffers and job tables are
fixed per group, the Adam step counter and group learning rates live in
device memory, and the freeze map / active list are read by the kernels when
they run. The scalar GSta logic (freeze-map actions, subset PSNR, early stop,
plateau learning rate) runs on the host between replays, per scene. A scene
that finishes leaves the batch and the graphs are captured again without it.

Nothing here computes: this module allocates buffers (PyTorch is the
allocator), fills the job tables and calls the C ABI.

  python -m paper_2504_06716_gb300.batch --steps 60      # timing of the four ways to run a step
"""
from __future__ import annotations

import argparse
import ctypes
import dataclasses
import json
import time

import numpy as np
import torch

from . import lib, pipeline, synth
from .autotune import retile
from .schedule import FREEZE_RESET, FREEZE_UPDATE, GStaConfig, GStaController, calibrate_eps0

SIZES = (50_000, 120_000, 250_000, 400_000, 600_000, 900_000, 1_400_000, 2_000_000)
RES = 800
VIEWS_PER_STEP = 4
N_VIEWS = 18  # every 8th held out: 16 training views = 4 groups of 4
# replayed graph / eager with parallel streams / eager on one stream / eager, one rasteriser launch per job
MODES = ("graph", "batched", "serial", "per_job")


def render_targets(scene: synth.Scene, cams, device) -> dict:
    """Target images of every camera, rendered from the scene's ground-truth set."""
    gtm = pipeline.Model(scene.gt, device=device, trainable=False)
    views = sorted(set(scene.train_views) | set(scene.test_views))
    gv = gtm.make_view(cams[views[0]], gtm.measure_capacity([cams[v] for v in views]), trainable=False)
    out = {}
    for v in views:
        gtm.retarget(gv, cams[v])
        gtm.rasterize(gv)
        out[v] = gv.image.clone()
    if lib.gs_get_device_error():
        raise RuntimeError("device error while rendering targets")
    return out


@dataclasses.dataclass
class Slot:
    """Buffers of one of a scene's views within a batch step."""
    view: pipeline.View
    splats: torch.Tensor
    grad2d: torch.Tensor


class BatchScene:
    """One scene of the batch: its model, controller and per-slot buffers."""

    def __init__(self, scene: synth.Scene, cfg: GStaConfig, tile: int, views_per_step: int, device, seed: int,
                 extent: float = 4.4, calibrate: bool = True):
        self.scene, self.cfg, self.device = scene, cfg, torch.device(device)
        self.cams = [lib.camera(c, tile=tile) for c in scene.cameras]
        self.targets = render_targets(scene, self.cams, self.device)
        self.model = pipeline.Model(scene.init, device=self.device)
        self.n = self.model.n
        self.lrs = pipeline.default_lrs(extent)
        self.ctrl = GStaController(cfg, self.lrs[0])
        self.lr_dev = torch.tensor(self.lrs, dtype=torch.float32, device=self.device)
        self.lr_host = list(self.lrs)
        self.step_dev = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.adam_scratch = torch.zeros(2, dtype=torch.float32, device=self.device)
        perm = [scene.train_views[i] for i in np.random.default_rng(seed).permutation(len(scene.train_views))]
        n_groups = len(perm) // views_per_step
        self.groups = [perm[g * views_per_step:(g + 1) * views_per_step] for g in range(n_groups)]
        H, W = self.cams[0].height, self.cams[0].width
        self.psnr_ws = torch.zeros(lib.gs_psnr_workspace_bytes(1, H, W), dtype=torch.uint8, device=self.device)
        self.psnr_out = torch.zeros(1, device=self.device)
        self.calibrate, self.calibrated = calibrate, False
        self.eps0 = (cfg.eps0_xyz, cfg.eps0_rgb)
        self.k = 0
        self.events: list[tuple[int, str, float]] = []
        self.slots: list[Slot] = []
        self.capacity = 0
        self.overflows = 0

    # ---- buffers ----
    def allocate(self, tile: int, capacity: int | None = None, slack: float = 1.25):
        self.cams = [retile(c, tile) for c in self.cams]
        m = self.model
        if capacity is None:
            capacity = m.measure_capacity([self.cams[v] for v in self.scene.train_views + self.scene.test_views],
                                          slack)
        self.capacity = capacity
        self.slots = []
        for i in range(len(self.groups[0])):
            # slot 0 shares the model's own splat and grad2d buffers
            splats = m.splats if i == 0 else torch.zeros_like(m.splats)
            grad2d = m.grad2d if i == 0 else torch.zeros_like(m.grad2d)
            self.slots.append(Slot(m.make_view(self.cams[self.groups[0][i]], capacity), splats, grad2d))

    def jobs(self, group: int) -> list[lib.GsRasterJob]:
        out = []
        for slot, v in zip(self.slots, self.groups[group]):
            vw = slot.view
            out.append(lib.GsRasterJob(slot.splats.data_ptr(), vw.vals.data_ptr(), vw.ranges.data_ptr(),
                                       vw.image.data_ptr(), vw.t_final.data_ptr(), vw.n_last.data_ptr(),
                                       vw.dl.data_ptr(), self.model.frozen.data_ptr(), slot.grad2d.data_ptr(),
                                       self.cams[v]))
        return out

    # ---- the device work of a step, split at the two batched launches ----
    def enqueue_front(self, group: int):
        m = self.model
        for slot, v in zip(self.slots, self.groups[group]):
            cam, vw = self.cams[v], slot.view
            lib.gs_project(m.P, m.n, m.sh_degree, cam, slot.splats)
            lib.gs_sort(slot.splats, m.n, cam, vw.sort_ws, vw.capacity, vw.vals, vw.ranges, vw.count)

    def enqueue_loss(self, group: int):
        for slot, v in zip(self.slots, self.groups[group]):
            vw, cam = slot.view, self.cams[v]
            lib.gs_loss(vw.image, self.targets[v], cam.height, cam.width, 0.2, vw.loss_ws, vw.loss, vw.dl)

    def enqueue_back(self, group: int):
        m = self.model
        for i, (slot, v) in enumerate(zip(self.slots, self.groups[group])):
            fn = lib.gs_project_bwd if i == 0 else lib.gs_project_bwd_accum
            fn(m.P, m.n, m.sh_degree, self.cams[v], slot.splats, m.act, m.n_active, slot.grad2d, m.G, m.acc_xyz,
               m.acc_rgb, m.cnt)
        lib.gs_adam_masked_devstep(m.P, m.G, m.m, m.v, m.n, m.act, m.n_active, self.lr_dev, 0.9, 0.999, 1e-15,
                                   self.step_dev, self.adam_scratch)

    def enqueue_per_job(self, group: int, fwd_cfg, bwd_cfg, backward: bool):
        """The rasteriser launches of this scene's jobs, one launch per job."""
        m = self.model
        for slot, v in zip(self.slots, self.groups[group]):
            vw, cam = slot.view, self.cams[v]
            if backward:
                lib.gs_raster_bwd_cfg(slot.splats, vw.vals, vw.ranges, cam, bwd_cfg, vw.t_final, vw.n_last, vw.dl,
                                      m.frozen, slot.grad2d)
            else:
                lib.gs_render_fwd_cfg(slot.splats, vw.vals, vw.ranges, cam, fwd_cfg, vw.image, vw.t_final,
                                      vw.n_last)

    # ---- host logic between steps (Algorithm 1's scalar part) ----
    def thresholds(self, k: int) -> tuple[float, float]:
        ex, er = self.ctrl.thresholds(k)
        return ex * self.eps0[0] / self.cfg.eps0_xyz, er * self.eps0[1] / self.cfg.eps0_rgb

    def psnr_of(self, views) -> float:
        m, vw = self.model, self.slots[0].view
        vals = []
        for v in views:
            m.retarget(vw, self.cams[v])
            m.rasterize(vw)
            lib.gs_psnr(vw.image, self.targets[v], 1, vw.cam.height, vw.cam.width, self.psnr_ws, self.psnr_out)
            vals.append(self.psnr_out.clone())
        return float(torch.stack(vals).mean().item())

    def before_step(self):
        """Freeze-map action, subset PSNR / early stop and the xyz rate for step k."""
        k, m, c = self.k, self.model, self.ctrl
        mode = c.freeze_mode(k)
        if mode is not None:
            if mode == FREEZE_UPDATE and self.calibrate and not self.calibrated:
                self.calibrated = True
                res = calibrate_eps0(self.cfg, c, k, m.acc_xyz.cpu().numpy(), m.acc_rgb.cpu().numpy(),
                                     m.cnt.cpu().numpy())
                if res is not None:
                    self.eps0 = res[0]
                    self.events.append((k, "calibrated", res[1]))
            ex, er = self.thresholds(k)
            m.freeze_update(ex, er, mode)
        if c.wants_psnr(k):
            p = self.psnr_of(self.scene.subset_views)
            self.events.append((k, "psnr", p))
            if c.report_psnr(k, p):
                m.freeze_update(0.0, 0.0, FREEZE_RESET)
                self.events.append((k, "early_stop", p))
        lr = c.lr_xyz_at(k)
        if lr != self.lr_host[0]:
            self.lr_host[0] = lr
            self.lr_dev[0].fill_(lr)

    def after_step(self):
        if self.ctrl.after_step(self.k):
            self.model.freeze_update(0.0, 0.0, FREEZE_RESET)
        self.k += 1

    def finished(self) -> bool:
        return self.ctrl.finished(self.k)

    def max_count(self) -> int:
        return max(int(s.view.count.item()) for s in self.slots)


class BatchTrainer:
    """All scenes of the batch, the job tables and the per-group CUDA graphs."""

    def __init__(self, scenes: list[synth.Scene], cfg: GStaConfig, tile: int = 16, views_per_step: int = VIEWS_PER_STEP,
                 fwd=None, bwd=None, device="cuda", calibrate: bool = True):
        self.device = torch.device(device)
        self.cfg = cfg
        self.scenes = [BatchScene(s, cfg, tile, views_per_step, self.device, seed=100 + i, calibrate=calibrate)
                       for i, s in enumerate(scenes)]
        self.n_groups = min(len(s.groups) for s in self.scenes)
        self.fwd, self.bwd = fwd, bwd  # (pixels per thread, batch) or None for the library defaults
        self.queue = torch.zeros(1, dtype=torch.int32, device=self.device)
        # largest scene first, so that its long chain of launches starts first
        self.scenes.sort(key=lambda s: -s.n)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in self.scenes]
        self.k = 0
        self.capacity_check_every = 100
        self.set_tile(tile)

    # ---- configuration ----
    def set_tile(self, tile: int, fwd=None, bwd=None):
        self.tile = tile
        if fwd is not None:
            self.fwd, self.bwd = fwd, bwd
        for s in self.scenes:
            s.allocate(tile)
        self._rebuild()

    def _rebuild(self):
        """Job tables of the scenes still training; drops every captured graph."""
        self.active = [s for s in self.scenes if not s.finished()]
        self.job_tables = []
        for g in range(self.n_groups):
            jobs = [j for s in self.active for j in s.jobs(g)]
            raw = (lib.GsRasterJob * max(len(jobs), 1))(*jobs)
            host = torch.frombuffer(bytearray(bytes(raw)), dtype=torch.uint8)
            self.job_tables.append((host.to(self.device), len(jobs)))
        self.graphs: dict[int, tuple[torch.cuda.CUDAGraph, int]] = {}

    def _cfg(self, which):
        v = self.fwd if which == "fwd" else self.bwd
        return None if v is None else lib.raster_config(*v)

    # ---- one step's device work ----
    def per_scene(self, fn, concurrent: bool = True):
        """fn(scene) for every active scene. Concurrent: each scene's work goes
        on a stream of its own, forked from and joined back into the current
        stream (captured, the forks become parallel branches of the graph), so
        the many small launches of the small scenes overlap instead of queueing
        behind one another."""
        if not concurrent:
            for s in self.active:
                fn(s)
            return
        main = torch.cuda.current_stream()
        for s, st in zip(self.active, self.streams):
            st.wait_stream(main)
            with torch.cuda.stream(st):
                fn(s)
        for st in self.streams[:len(self.active)]:
            main.wait_stream(st)

    def enqueue(self, group: int, mode: str = "batched"):
        """The device work of one batch step. mode: "batched" -- the two
        persistent launches and per-scene work on parallel streams; "serial" --
        the same launches, all on one stream; "per_job" -- one stream and one
        rasteriser launch per (scene, view) job."""
        table, n_jobs = self.job_tables[group]
        cam = self.active[0].cams[0]
        conc = mode == "batched"
        self.per_scene(lambda s: s.enqueue_front(group), conc)
        if mode == "per_job":
            self.per_scene(lambda s: s.enqueue_per_job(group, self._cfg("fwd"), None, backward=False), False)
        else:
            lib.gs_render_fwd_batch(table, n_jobs, cam.width, cam.height, self.tile, self._cfg("fwd"), self.queue)
        self.per_scene(lambda s: s.enqueue_loss(group), conc)
        if mode == "per_job":
            self.per_scene(lambda s: s.enqueue_per_job(group, None, self._cfg("bwd"), backward=True), False)
        else:
            lib.gs_raster_bwd_batch(table, n_jobs, cam.width, cam.height, self.tile, self._cfg("bwd"), self.queue)
        self.per_scene(lambda s: s.enqueue_back(group), conc)

    def _graph(self, group: int):
        if group not in self.graphs:
            n0 = lib.gs_launch_count()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self.enqueue(group, "batched")
            self.graphs[group] = (g, lib.gs_launch_count() - n0)
        return self.graphs[group]

    # ---- training ----
    def group_of(self, k: int) -> int:
        return k % self.n_groups

    def step(self, mode: str = "graph") -> int:
        """One batch step; returns the number of library kernels it launched."""
        for s in self.active:
            s.before_step()
        group = self.group_of(self.k)
        if mode == "graph":
            if group not in self.graphs:
                n0 = lib.gs_launch_count()
                self.enqueue(group, "batched")  # this step runs eagerly; later ones replay the capture
                launches = lib.gs_launch_count() - n0
                self._graph(group)
            else:
                g, launches = self.graphs[group]
                g.replay()
        else:
            n0 = lib.gs_launch_count()
            self.enqueue(group, mode)
            launches = lib.gs_launch_count() - n0
        for s in self.active:
            s.after_step()
        self.k += 1
        if self.k % self.capacity_check_every == 0:
            self.check_capacity()
        if any(s.finished() for s in self.active):
            self._rebuild()
        return launches

    def check_capacity(self, headroom: float = 0.8, grow: float = 1.5):
        flags = lib.gs_get_device_error()
        if flags & ~lib.GS_FLAG_CAPACITY:
            raise RuntimeError(f"device error flags {flags:#x} at batch step {self.k}")
        changed = False
        for s in self.active:
            P = s.max_count()
            if flags & lib.GS_FLAG_CAPACITY and P > s.capacity:
                s.overflows += 1
                s.events.append((s.k, "capacity_overflow", float(P)))
            if P > headroom * s.capacity:
                s.allocate(self.tile, int(max(P, s.capacity) * grow) + 1024)
                s.events.append((s.k, "capacity", float(s.capacity)))
                changed = True
        if changed:
            self._rebuild()

    def finished(self) -> bool:
        return not self.active

    def gaussian_views_per_step(self) -> int:
        return sum(s.n * len(s.groups[0]) for s in self.active)


# ---- autotuner for the batched launches ----
def _time(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(bt: BatchTrainer, tiles=(8, 16, 32), ppts=(1, 2, 4), batches=(32, 64, 128, 256), reps: int = 3) -> dict:
    """Pick the tile size (8/16/32) and the (pixels per thread, splats per
    shared-memory batch) of the two persistent launches by timing them on the
    trainer's own scenes, for view group 0. Tile size moves work between the
    sort and the rasteriser, so the choice minimises projection + sort + best
    forward + best backward. Runs real training steps (one per tile)."""
    table, best = {}, None
    all_ppts = ppts
    for tile in tiles:
        ppts = [p for p in all_ppts if tile * tile // p >= 32]  # whole warps per tile
        bt.set_tile(tile)
        bt.step("batched")  # fills every buffer for group 0 (and advances training one step)
        tbl, n_jobs = bt.job_tables[0]
        H, W = bt.active[0].cams[0].height, bt.active[0].cams[0].width
        t_front = _time(lambda: bt.per_scene(lambda s: s.enqueue_front(0)), reps)
        fwd_t, bwd_t = {}, {}
        for ppt in ppts:
            for b in batches:
                c = lib.raster_config(ppt, b)
                fwd_t[(ppt, b)] = _time(lambda: lib.gs_render_fwd_batch(tbl, n_jobs, W, H, tile, c, bt.queue), reps)
        for ppt in ppts:
            for b in batches:
                c = lib.raster_config(ppt, b)
                bwd_t[(ppt, b)] = _time(lambda: lib.gs_raster_bwd_batch(tbl, n_jobs, W, H, tile, c, bt.queue), reps)
        for s in bt.active:
            for slot in s.slots:
                slot.grad2d.zero_()
        bf, bb = min(fwd_t, key=fwd_t.get), min(bwd_t, key=bwd_t.get)
        total = t_front + fwd_t[bf] + bwd_t[bb]
        table[tile] = dict(project_sort_ms=t_front, fwd_ms={f"{p}x{b}": t for (p, b), t in fwd_t.items()},
                           bwd_ms={f"{p}x{b}": t for (p, b), t in bwd_t.items()}, best_fwd=bf, best_bwd=bb,
                           total_ms=total)
        if best is None or total < best[0]:
            best = (total, tile, bf, bb)
    bt.set_tile(best[1], best[2], best[3])
    return dict(tile=best[1], fwd=best[2], bwd=best[3], table=table)


def make_scenes(sizes=SIZES, res: int = RES, n_views: int = N_VIEWS, seed: int = 40) -> list[synth.Scene]:
    """The batch's scenes: surface scenes of the given sizes, ground truth of the same size."""
    return [synth.surface_scene(n, n, n_views, res, res, seed=seed + 2 * i) for i, n in enumerate(sizes)]


def measure(bt: BatchTrainer, steps: int, warmup: int, mode: str) -> dict:
    """Average device time of ``steps`` batch steps (after ``warmup``), CUDA
    events on the launching stream."""
    launches = 0
    for _ in range(warmup):
        bt.step(mode)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record()
    for _ in range(steps):
        launches += bt.step(mode)
    e1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = e0.elapsed_time(e1) / steps
    return dict(mode=mode, ms_per_step=ms, wall_ms_per_step=1e3 * wall / steps, launches_per_step=launches / steps,
                gaussian_views_per_s=bt.gaussian_views_per_step() / (ms * 1e-3))


def main():
    ap = argparse.ArgumentParser(description="batched uneven-scene training: graph vs eager vs per-job launches")
    ap.add_argument("--sizes", default=",".join(str(s) for s in SIZES))
    ap.add_argument("--res", type=int, default=RES)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=8)
    ap.add_argument("--pretrain", type=int, default=3200, help="steps before timing (into the freezing window)")
    ap.add_argument("--no-tune", action="store_true")
    args = ap.parse_args()
    torch.cuda.set_device(0)
    sizes = [int(x) for x in args.sizes.split(",")]
    t0 = time.perf_counter()
    bt = BatchTrainer(make_scenes(sizes, args.res), GStaConfig())
    setup_s = time.perf_counter() - t0
    tuning = None if args.no_tune else tune(bt)
    for _ in range(args.pretrain):
        bt.step("graph")
    out = dict(workload=f"batch-8-scenes-{args.res}x{args.res}", sizes=sizes, views_per_step=VIEWS_PER_STEP,
               setup_s=setup_s, tuning=tuning, pretrain_steps=args.pretrain,
               active_fraction=[float(s.model.n_active.item()) / s.n for s in bt.active])
    for mode in MODES:
        out[mode] = measure(bt, args.steps, args.warmup, mode)
    out["graph_speedup_vs_per_job"] = out["per_job"]["ms_per_step"] / out["graph"]["ms_per_step"]
    out["graph_speedup_vs_serial"] = out["serial"]["ms_per_step"] / out["graph"]["ms_per_step"]
    out["events"] = {s.n: [e for e in s.events if e[1] != "psnr"] for s in bt.scenes}
    if lib.gs_get_device_error():
        raise RuntimeError("device error flags raised during the run")
    print(json.dumps(out, default=str))


if __name__ == "__main__":
    main()
