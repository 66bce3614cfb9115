"""Autotuner for the rasteriser launch shape.

Times, on the caller's own model and views, every tile size (8, 16, 32) with
every pixels-per-thread (1, 2, 4 where a tile fills whole warps) and batch size (32, 64, 128, 256) of the two
rasteriser kernels, and picks the tile size whose projection + sort + best
forward + best backward is fastest. Results depend only on timing: every
shape computes the same image and, up to atomic reordering, the same
gradients.
"""
from __future__ import annotations

import dataclasses
import json

import torch

from . import lib


@dataclasses.dataclass
class RasterTuning:
    tile: int
    fwd: tuple[int, int]  # (pixels per thread, batch)
    bwd: tuple[int, int]
    table: dict

    def to_json(self) -> str:
        return json.dumps(dataclasses.asdict(self))


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


def retile(cam: lib.GsCamera, tile: int) -> lib.GsCamera:
    c = lib.GsCamera()
    ctypes_copy = bytes(memoryview(cam).cast("B"))
    memoryview(c).cast("B")[:] = ctypes_copy
    c.tile = tile
    return c


def tune(model, cams, targets, tiles=(8, 16, 32), ppts=(1, 2, 4), batches=(32, 64, 128, 256), reps: int = 3,
         n_views: int = 2) -> RasterTuning:
    """``cams``/``targets``: a few representative views (camera, target image)."""
    table = {}
    best = None
    all_ppts = ppts
    for tile in tiles:
        ppts = [p for p in all_ppts if tile * tile // p >= 32]  # whole warps per tile
        views = [retile(c, tile) for c in cams[:n_views]]
        cap = model.measure_capacity(views)
        v = model.make_view(views[0], cap)
        t_ps = t_f = t_b = 0.0
        fwd_times, bwd_times = {}, {}
        for cam, gt in zip(views, targets[:n_views]):
            model.retarget(v, cam)
            t_ps += _time(lambda: (lib.gs_project(model.P, model.n, model.sh_degree, v.cam, model.splats),
                                   lib.gs_sort(model.splats, model.n, v.cam, v.sort_ws, v.capacity, v.vals, v.ranges,
                                               v.count)), reps)
            for ppt in ppts:
                for b in batches:
                    cfg = lib.raster_config(ppt, b)
                    fwd_times[(ppt, b)] = fwd_times.get((ppt, b), 0.0) + _time(
                        lambda: model.render_fwd(v, cfg), reps)
            model.loss(v, gt)
            for ppt in ppts:
                for b in batches:
                    cfg = lib.raster_config(ppt, b)
                    bwd_times[(ppt, b)] = bwd_times.get((ppt, b), 0.0) + _time(
                        lambda: model.raster_bwd(v, cfg), reps)
        model.grad2d.zero_()
        bf = min(fwd_times, key=fwd_times.get)
        bb = min(bwd_times, key=bwd_times.get)
        total = t_ps + fwd_times[bf] + bwd_times[bb]
        table[tile] = dict(project_sort_ms=t_ps / n_views, fwd_ms={f"{k[0]}x{k[1]}": t / n_views
                                                                  for k, t in fwd_times.items()},
                           bwd_ms={f"{k[0]}x{k[1]}": t / n_views for k, t in bwd_times.items()},
                           best_fwd=bf, best_bwd=bb, total_ms=total / n_views)
        if best is None or total < best[0]:
            best = (total, tile, bf, bb)
        del v
    return RasterTuning(tile=best[1], fwd=best[2], bwd=best[3], table=table)
