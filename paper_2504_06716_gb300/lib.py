"""Thin ctypes binding of ``libgsta.so`` (declared in ``include/gsta.h``).

Argument marshalling only: every function here takes torch tensors (or raw
integers), checks dtype/device/contiguity, and passes ``data_ptr()`` values
and the current CUDA stream to the C entry point of the same name. All
arithmetic runs in the CUDA kernels behind the C ABI. A missing library or a
non-zero status raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgsta.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "gsta.h")

ROW = 64       # floats per parameter row
SPLAT = 12     # floats per splat record
GRAD2D = 12    # floats per raster-gradient row

GS_FLAG_CAPACITY, GS_FLAG_NONFINITE, GS_FLAG_TIMEOUT, GS_FLAG_BADJOB = 1, 2, 4, 8


class GsError(RuntimeError):
    def __init__(self, name: str, status: int, text: str):
        super().__init__(f"{name} failed: {text} (status {status})")
        self.status = status


class GsRasterConfig(ctypes.Structure):
    _fields_ = [("pixels_per_thread", ctypes.c_int32), ("batch", ctypes.c_int32)]


def raster_config(pixels_per_thread: int, batch: int) -> GsRasterConfig:
    c = GsRasterConfig()
    c.pixels_per_thread, c.batch = int(pixels_per_thread), int(batch)
    return c


class GsCamera(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("tile", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
        ("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("campos", ctypes.c_float * 3),
        ("znear", ctypes.c_float), ("dilation", ctypes.c_float), ("bg", ctypes.c_float * 3),
    ]

    @property
    def tiles_x(self) -> int:
        return (self.width + self.tile - 1) // self.tile

    @property
    def tiles(self) -> int:
        return self.tiles_x * ((self.height + self.tile - 1) // self.tile)


def camera(cam, tile: int = 16, znear: float = 0.2, dilation: float = 0.3, bg=(0.0, 0.0, 0.0)) -> GsCamera:
    """A ``GsCamera`` from any object with width, height, fx, fy, cx, cy, R, t, campos."""
    c = GsCamera()
    c.width, c.height, c.tile = int(cam.width), int(cam.height), int(tile)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.R[:] = [float(v) for v in np.asarray(cam.R, np.float64).reshape(9)]
    c.t[:] = [float(v) for v in np.asarray(cam.t, np.float64).reshape(3)]
    c.campos[:] = [float(v) for v in np.asarray(cam.campos, np.float64).reshape(3)]
    c.znear, c.dilation = float(znear), float(dilation)
    c.bg[:] = [float(v) for v in bg]
    return c


_P = ctypes.c_void_p
_I64, _I32, _F32, _SZ, _U32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_size_t, ctypes.c_uint32
_CAM = ctypes.POINTER(GsCamera)

_SIGS = {
    "gs_project": ([_P, _I64, _I32, _CAM, _P, _P], _I32),
    "gs_sort_workspace_bytes": ([_I64, _I64, _I32, _I32, _I32], _SZ),
    "gs_sort": ([_P, _I64, _CAM, _P, _SZ, _I64, _P, _P, _P, _P], _I32),
    "gs_render_fwd": ([_P, _P, _P, _CAM, _P, _P, _P, _P], _I32),
    "gs_render_fwd_cfg": ([_P, _P, _P, _CAM, ctypes.POINTER(GsRasterConfig), _P, _P, _P, _P], _I32),
    "gs_raster_bwd_cfg": ([_P, _P, _P, _CAM, ctypes.POINTER(GsRasterConfig), _P, _P, _P, _P, _P, _P], _I32),
    "gs_render_fwd_resume": ([_P, _P, _P, _CAM, ctypes.POINTER(GsRasterConfig), _P, _P, _P, _P, _P, _P, _P], _I32),
    "gs_raster_bwd_resume": ([_P, _P, _P, _CAM, ctypes.POINTER(GsRasterConfig), _P, _P, _P, _P, _P, _P, _P, _P],
                             _I32),
    "gs_loss_workspace_bytes": ([_I32, _I32], _SZ),
    "gs_loss": ([_P, _P, _I32, _I32, _F32, _P, _SZ, _P, _P, _P], _I32),
    "gs_raster_bwd": ([_P, _P, _P, _CAM, _P, _P, _P, _P, _P, _P], _I32),
    "gs_project_bwd": ([_P, _I64, _I32, _CAM, _P, _P, _P, _P, _P, _P, _P, _P, _P], _I32),
    "gs_project_bwd_accum": ([_P, _I64, _I32, _CAM, _P, _P, _P, _P, _P, _P, _P, _P, _P], _I32),
    "gs_render_fwd_batch": ([_P, _I32, _I32, _I32, _I32, ctypes.POINTER(GsRasterConfig), _P, _P], _I32),
    "gs_raster_bwd_batch": ([_P, _I32, _I32, _I32, _I32, ctypes.POINTER(GsRasterConfig), _P, _P], _I32),
    "gs_render_bwd": ([_P, _I64, _I32, _CAM, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P], _I32),
    "gs_freeze_workspace_bytes": ([_I64], _SZ),
    "gs_freeze_update": ([_I64, _P, _P, _P, _P, _F32, _F32, _I32, _P, _P, _P, _SZ, _P], _I32),
    "gs_freeze_update_noalloc": ([_I64, _P, _P, _P, _P, _F32, _F32, _I32, _P, _P, _P], _I32),
    "gs_adam_masked": ([_P, _P, _P, _P, _I64, _P, _P, ctypes.POINTER(ctypes.c_float), _F32, _F32, _F32, _I64, _P],
                       _I32),
    "gs_pred_history": ([_I64, _P, _P, _P, _P, _P, _P], _I32),
    "gs_pred_features": ([_I64, _P, _P, _P, _P, _P, _I32, _I32, _F32, _F32, _P, _P], _I32),
    "gs_mlp_fwd": ([_I64, _P, _P, _P, _P, _P], _I32),
    "gs_mlp_grad": ([_I64, _P, _P, _P, _F32, _P, _P, _P, _P, _P], _I32),
    "gs_mlp_adam": ([_P, _P, _P, _P, _P, _F32, _F32, _F32, _F32, _I64, _P], _I32),
    "gs_mlp_refresh": ([_P, _P, _P], _I32),
    "gs_freeze_apply": ([_I64, _P, _F32, _P, _P, _P, _P, _SZ, _P], _I32),
    "gs_freeze_select_workspace_bytes": ([_I64], _SZ),
    "gs_freeze_select": ([_I64, _P, _P, _P, _P, _F32, _F32, _I32, _F32, _P, _P, _P, _P, _SZ, _P], _I32),
    "gs_adam_masked_devstep": ([_P, _P, _P, _P, _I64, _P, _P, _P, _F32, _F32, _F32, _P,
                                _P, _P], _I32),
    "gs_raster_pair_counts": ([_P, _P, _P, _CAM, _P, _P, _P, _P], _I32),
    "gs_project_bwd_stats": ([_P, _I64, _I32, _CAM, _P, _P, _P, _P, _P, _I32, _P, _I32, _P], _I32),
    "gs_densify_workspace_bytes": ([_I64], _SZ),
    "gs_densify_plan": ([_I64, _P, _P, _P, _P, _SZ, _P, _P], _I32),
    "gs_densify_apply": ([_I64, _P, _P, _P, _P, _P, _I32, _P, _P, _P, _SZ, _I64, _P, _P, _P, _P, _P], _I32),
    "gs_opacity_reset": ([_I64, _P, _P, _P, _F32, _P], _I32),
    "gs_opacity_to_abs": ([_I64, _P, _P, _P, _I32, _P, _P], _I32),
    "gs_train_step": ([_P, _P, _P, _P, _I64, _P], _I32),
    "gs_hit_counts": ([_P, _P, _P, _CAM, _P, _P, _P], _I32),
    "gs_significance_workspace_bytes": ([_I64], _SZ),
    "gs_significance_mark": ([_I64, _P, _P, _I32, _F32, _F32, _F32, _P, _P, _SZ, _P], _I32),
    "gs_resize_area": ([_P, _I32, _I32, _I32, _P, _I32, _I32, _P], _I32),
    "gs_blur": ([_P, _I32, _I32, _I32, _F32, _P, _P], _I32),
    "gs_project_ex": ([_P, _I64, _I32, _I32, _P, _P, _P], _I32),
    "gs_project_bwd_ex": ([_P, _I64, _I32, _I32, _F32, _P, _P, _P, _P, _P, _P, _I32, _P, _I32, _P], _I32),
    "gs_adam_masked_groups": ([_P, _P, _P, _P, _I64, _P, _P, _P, _I32, _F32, _F32, _F32, _I64, _P], _I32),
    "gs_psnr_workspace_bytes": ([_I32, _I32, _I32], _SZ),
    "gs_psnr": ([_P, _P, _I32, _I32, _I32, _P, _SZ, _P, _P], _I32),
    "gs_get_device_error": ([ctypes.POINTER(ctypes.c_uint32), _P], _I32),
    "gs_status_string": ([_I32], ctypes.c_char_p),
    "gs_launch_count": ([], ctypes.c_uint64),
    "gs_version": ([], _I32),
}

_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library missing: {LIB_PATH} (run __graft_entry__.build())")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(name: str, status: int):
    if status != 0:
        raise GsError(name, status, load().gs_status_string(status).decode())


def _ptr(t, dtype=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch

    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return t.data_ptr()


def _stream(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


# ---------------------------------------------------------------- entry points (same names as the C ABI)


def gs_project(P, n: int, sh_degree: int, cam: GsCamera, splats, stream=None):
    import torch

    _check("gs_project", load().gs_project(_ptr(P, torch.float32, "P"), n, sh_degree, ctypes.byref(cam),
                                           _ptr(splats, torch.float32, "splats"), _stream(stream)))


GS_OPACITY_SIGMOID, GS_OPACITY_ABS, GS_VOLUME_MASK = 0, 1, 2


def gs_project_ex(P, n: int, sh_degree: int, opacity_act: int, cam: GsCamera, splats, stream=None):
    import torch

    _check("gs_project_ex", load().gs_project_ex(_ptr(P, torch.float32, "P"), n, sh_degree, opacity_act,
                                                 ctypes.byref(cam), _ptr(splats, torch.float32, "splats"),
                                                 _stream(stream)))


def gs_sort_workspace_bytes(n: int, capacity: int, cam: GsCamera) -> int:
    return int(load().gs_sort_workspace_bytes(n, capacity, cam.width, cam.height, cam.tile))


def gs_sort(splats, n: int, cam: GsCamera, ws, capacity: int, vals, ranges, count, stream=None):
    import torch

    _check("gs_sort", load().gs_sort(_ptr(splats, torch.float32, "splats"), n, ctypes.byref(cam),
                                     _ptr(ws, torch.uint8, "ws"), ws.numel(), capacity,
                                     _ptr(vals, torch.int32, "vals"), _ptr(ranges, torch.int32, "ranges"),
                                     _ptr(count, torch.int64, "count"), _stream(stream)))


def gs_render_fwd(splats, vals, ranges, cam: GsCamera, image, t_final, n_last, stream=None):
    import torch

    _check("gs_render_fwd", load().gs_render_fwd(_ptr(splats, torch.float32, "splats"), _ptr(vals, torch.int32, "vals"),
                                                 _ptr(ranges, torch.int32, "ranges"), ctypes.byref(cam),
                                                 _ptr(image, torch.float32, "image"),
                                                 _ptr(t_final, torch.float32, "t_final"),
                                                 _ptr(n_last, torch.int32, "n_last"), _stream(stream)))


def gs_render_fwd_cfg(splats, vals, ranges, cam: GsCamera, cfg, image, t_final, n_last, stream=None):
    import torch

    _check("gs_render_fwd_cfg", load().gs_render_fwd_cfg(
        _ptr(splats, torch.float32, "splats"), _ptr(vals, torch.int32, "vals"), _ptr(ranges, torch.int32, "ranges"),
        ctypes.byref(cam), None if cfg is None else ctypes.byref(cfg), _ptr(image, torch.float32, "image"),
        _ptr(t_final, torch.float32, "t_final"), _ptr(n_last, torch.int32, "n_last"), _stream(stream)))


def _resume_sizes(cam: GsCamera, resume, resume_pos):
    """The resume record's sizes: [H][W][4] float and [tiles] int32."""
    if resume is not None and resume.numel() < 4 * cam.width * cam.height:
        raise ValueError("resume holds fewer than H * W * 4 floats")
    if resume_pos is not None and resume_pos.numel() < cam.tiles:
        raise ValueError("resume_pos holds fewer than tiles entries")


def gs_render_fwd_resume(splats, vals, ranges, cam: GsCamera, cfg, frozen, image, t_final, n_last, resume,
                         resume_pos, stream=None):
    import torch

    _resume_sizes(cam, resume, resume_pos)
    _check("gs_render_fwd_resume", load().gs_render_fwd_resume(
        _ptr(splats, torch.float32, "splats"), _ptr(vals, torch.int32, "vals"), _ptr(ranges, torch.int32, "ranges"),
        ctypes.byref(cam), None if cfg is None else ctypes.byref(cfg), _ptr(frozen, torch.uint8, "frozen"),
        _ptr(image, torch.float32, "image"), _ptr(t_final, torch.float32, "t_final"),
        _ptr(n_last, torch.int32, "n_last"), _ptr(resume, torch.float32, "resume"),
        _ptr(resume_pos, torch.int32, "resume_pos"), _stream(stream)))


def gs_raster_bwd_resume(splats, vals, ranges, cam: GsCamera, cfg, t_final, n_last, dl_dimage, frozen, resume,
                         resume_pos, grad2d, stream=None):
    import torch

    _resume_sizes(cam, resume, resume_pos)
    _check("gs_raster_bwd_resume", load().gs_raster_bwd_resume(
        _ptr(splats, torch.float32, "splats"), _ptr(vals, torch.int32, "vals"), _ptr(ranges, torch.int32, "ranges"),
        ctypes.byref(cam), None if cfg is None else ctypes.byref(cfg), _ptr(t_final, torch.float32, "t_final"),
        _ptr(n_last, torch.int32, "n_last"), _ptr(dl_dimage, torch.float32, "dl_dimage"),
        _ptr(frozen, torch.uint8, "frozen"), _ptr(resume, torch.float32, "resume"),
        _ptr(resume_pos, torch.int32, "resume_pos"), _ptr(grad2d, torch.float32, "grad2d"), _stream(stream)))


def gs_raster_bwd_cfg(splats, vals, ranges, cam: GsCamera, cfg, t_final, n_last, dl_dimage, frozen, grad2d,
                      stream=None):
    import torch

    _check("gs_raster_bwd_cfg", load().gs_raster_bwd_cfg(
        _ptr(splats, torch.float32, "splats"), _ptr(vals, torch.int32, "vals"), _ptr(ranges, torch.int32, "ranges"),
        ctypes.byref(cam), None if cfg is None else ctypes.byref(cfg), _ptr(t_final, torch.float32, "t_final"),
        _ptr(n_last, torch.int32, "n_last"), _ptr(dl_dimage, torch.float32, "dl_dimage"),
        _ptr(frozen, torch.uint8, "frozen"), _ptr(grad2d, torch.float32, "grad2d"), _stream(stream)))


def gs_loss_workspace_bytes(H: int, W: int) -> int:
    return int(load().gs_loss_workspace_bytes(H, W))


def gs_loss(image, gt, H: int, W: int, lam: float, ws, loss, dl_dimage, stream=None):
    import torch

    _check("gs_loss", load().gs_loss(_ptr(image, torch.float32, "image"), _ptr(gt, torch.float32, "gt"), H, W, lam,
                                     _ptr(ws, torch.uint8, "ws"), ws.numel(), _ptr(loss, torch.float32, "loss"),
                                     _ptr(dl_dimage, torch.float32, "dl_dimage"), _stream(stream)))


def gs_raster_bwd(splats, vals, ranges, cam: GsCamera, t_final, n_last, dl_dimage, frozen, grad2d, stream=None):
    import torch

    _check("gs_raster_bwd", load().gs_raster_bwd(
        _ptr(splats, torch.float32, "splats"), _ptr(vals, torch.int32, "vals"), _ptr(ranges, torch.int32, "ranges"),
        ctypes.byref(cam), _ptr(t_final, torch.float32, "t_final"), _ptr(n_last, torch.int32, "n_last"),
        _ptr(dl_dimage, torch.float32, "dl_dimage"), _ptr(frozen, torch.uint8, "frozen"),
        _ptr(grad2d, torch.float32, "grad2d"), _stream(stream)))


def gs_project_bwd(P, n: int, sh_degree: int, cam: GsCamera, splats, act, n_active, grad2d, G, acc_xyz=None,
                   acc_rgb=None, cnt=None, stream=None):
    import torch

    _check("gs_project_bwd", load().gs_project_bwd(
        _ptr(P, torch.float32, "P"), n, sh_degree, ctypes.byref(cam), _ptr(splats, torch.float32, "splats"),
        _ptr(act, torch.int32, "act"), _ptr(n_active, torch.int32, "n_active"), _ptr(grad2d, torch.float32, "grad2d"),
        _ptr(G, torch.float32, "G"), _ptr(acc_xyz, torch.float32, "acc_xyz"), _ptr(acc_rgb, torch.float32, "acc_rgb"),
        _ptr(cnt, torch.int32, "cnt"), _stream(stream)))


def gs_project_bwd_accum(P, n: int, sh_degree: int, cam: GsCamera, splats, act, n_active, grad2d, G, acc_xyz=None,
                         acc_rgb=None, cnt=None, stream=None):
    import torch

    _check("gs_project_bwd_accum", load().gs_project_bwd_accum(
        _ptr(P, torch.float32, "P"), n, sh_degree, ctypes.byref(cam), _ptr(splats, torch.float32, "splats"),
        _ptr(act, torch.int32, "act"), _ptr(n_active, torch.int32, "n_active"), _ptr(grad2d, torch.float32, "grad2d"),
        _ptr(G, torch.float32, "G"), _ptr(acc_xyz, torch.float32, "acc_xyz"), _ptr(acc_rgb, torch.float32, "acc_rgb"),
        _ptr(cnt, torch.int32, "cnt"), _stream(stream)))


class GsGradStats(ctypes.Structure):
    _fields_ = [("acc_xyz", ctypes.c_void_p), ("acc_rgb", ctypes.c_void_p), ("cnt", ctypes.c_void_p),
                ("max_radius", ctypes.c_void_p)]


class GsStep(ctypes.Structure):
    """gs_step: every buffer of one training step (raw device pointers; the
    caller keeps the tensors alive while the struct is used)."""
    _fields_ = [
        ("P", ctypes.c_void_p), ("G", ctypes.c_void_p), ("m", ctypes.c_void_p), ("v", ctypes.c_void_p),
        ("splats", ctypes.c_void_p), ("grad2d", ctypes.c_void_p), ("n", ctypes.c_int64),
        ("sh_degree", ctypes.c_int32), ("opacity_act", ctypes.c_int32), ("mask_loss", ctypes.c_float),
        ("n_lr", ctypes.c_int32), ("frozen", ctypes.c_void_p),
        ("act", ctypes.c_void_p), ("n_active_dev", ctypes.c_void_p), ("stats", GsGradStats * 2),
        ("n_stats", ctypes.c_int32), ("sort_ws", ctypes.c_void_p), ("sort_ws_bytes", ctypes.c_size_t),
        ("capacity", ctypes.c_int64), ("vals", ctypes.c_void_p), ("ranges", ctypes.c_void_p),
        ("count_dev", ctypes.c_void_p), ("image", ctypes.c_void_p), ("t_final", ctypes.c_void_p),
        ("n_last", ctypes.c_void_p), ("dl_dimage", ctypes.c_void_p), ("loss_ws", ctypes.c_void_p),
        ("loss_ws_bytes", ctypes.c_size_t), ("loss_dev", ctypes.c_void_p), ("lambda_ssim", ctypes.c_float),
        ("fwd", GsRasterConfig), ("bwd", GsRasterConfig), ("b1", ctypes.c_float), ("b2", ctypes.c_float),
        ("eps", ctypes.c_float), ("bwd_events", ctypes.c_void_p * 2), ("resume", ctypes.c_void_p),
        ("resume_pos", ctypes.c_void_p),
    ]


def step_args(P, G, m, v, splats, grad2d, n: int, sh_degree: int, opacity_act: int, frozen, act, n_active, stats,
              sort_ws, capacity: int, vals, ranges, count, image, t_final, n_last, dl, loss_ws, loss, lam: float = 0.2,
              fwd=None, bwd=None, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-15, mask_loss: float = 0.0,
              n_lr: int = 6, resume=None, resume_pos=None) -> GsStep:
    """A gs_step for gs_train_step (tensors checked here once; the caller keeps them alive)."""
    import torch

    s = GsStep()
    f32, i32, u8 = torch.float32, torch.int32, torch.uint8
    s.P, s.G, s.m, s.v = (_ptr(t, f32, k) for t, k in ((P, "P"), (G, "G"), (m, "m"), (v, "v")))
    s.splats, s.grad2d = _ptr(splats, f32, "splats"), _ptr(grad2d, f32, "grad2d")
    s.n, s.sh_degree, s.opacity_act = int(n), int(sh_degree), int(opacity_act)
    s.mask_loss, s.n_lr = float(mask_loss), int(n_lr)
    s.frozen, s.act, s.n_active_dev = _ptr(frozen, u8, "frozen"), _ptr(act, i32, "act"), _ptr(n_active, i32, "n_active")
    if len(stats) > 2:
        raise ValueError("at most two statistics windows")
    for k, st in enumerate(stats):
        s.stats[k] = st
    s.n_stats = len(stats)
    s.sort_ws, s.sort_ws_bytes, s.capacity = _ptr(sort_ws, u8, "sort_ws"), sort_ws.numel(), int(capacity)
    s.vals, s.ranges = _ptr(vals, i32, "vals"), _ptr(ranges, i32, "ranges")
    s.count_dev = _ptr(count, torch.int64, "count")
    s.image, s.t_final, s.n_last = _ptr(image, f32, "image"), _ptr(t_final, f32, "t_final"), _ptr(n_last, i32, "n_last")
    s.dl_dimage = _ptr(dl, f32, "dl")
    s.loss_ws, s.loss_ws_bytes, s.loss_dev = _ptr(loss_ws, u8, "loss_ws"), loss_ws.numel(), _ptr(loss, f32, "loss")
    s.lambda_ssim = lam
    s.fwd = fwd if fwd is not None else GsRasterConfig(0, 0)
    s.bwd = bwd if bwd is not None else GsRasterConfig(0, 0)
    s.b1, s.b2, s.eps = b1, b2, eps
    if (resume is None) != (resume_pos is None):
        raise ValueError("resume and resume_pos go together")
    if resume is not None and (resume.numel() < 4 * t_final.numel() or 2 * resume_pos.numel() < ranges.numel()):
        raise ValueError("the resume record is [H][W][4] float and [tiles] int32")
    s.resume, s.resume_pos = _ptr(resume, f32, "resume"), _ptr(resume_pos, i32, "resume_pos")
    return s


def gs_train_step(step: GsStep, cam: GsCamera, gt, lr, adam_step: int, stream=None):
    import torch

    if len(lr) != (step.n_lr or 6):
        raise ValueError(f"gs_train_step wants {step.n_lr or 6} learning rates, got {len(lr)}")
    lr6 = (ctypes.c_float * len(lr))(*[float(x) for x in lr])
    _check("gs_train_step", load().gs_train_step(ctypes.byref(step), ctypes.byref(cam), _ptr(gt, torch.float32, "gt"),
                                                 lr6, adam_step, _stream(stream)))


GS_BLUR_SIGMA_MIN = float(np.float32(0.1))  # gs_blur copies below this (float32 comparison)


def gs_hit_counts(splats, vals, ranges, cam: GsCamera, n_last, hits, stream=None):
    import torch

    _check("gs_hit_counts", load().gs_hit_counts(
        _ptr(splats, torch.float32, "splats"), _ptr(vals, torch.int32, "vals"), _ptr(ranges, torch.int32, "ranges"),
        ctypes.byref(cam), _ptr(n_last, torch.int32, "n_last"), _ptr(hits, torch.int32, "hits"), _stream(stream)))


def gs_significance_workspace_bytes(n: int) -> int:
    return int(load().gs_significance_workspace_bytes(n))


def gs_significance_mark(n: int, P, hits, opacity_act: int, beta: float, quantile: float, fraction: float, mark, ws,
                         stream=None):
    import torch

    _check("gs_significance_mark", load().gs_significance_mark(
        n, _ptr(P, torch.float32, "P"), _ptr(hits, torch.int32, "hits"), opacity_act, beta, quantile, fraction,
        _ptr(mark, torch.uint8, "mark"), _ptr(ws, torch.uint8, "ws"), ws.numel(), _stream(stream)))


def gs_resize_area(src, C: int, W: int, H: int, dst, W2: int, H2: int, stream=None):
    import torch

    _check("gs_resize_area", load().gs_resize_area(_ptr(src, torch.float32, "src"), C, W, H,
                                                   _ptr(dst, torch.float32, "dst"), W2, H2, _stream(stream)))


def gs_blur(src, C: int, W: int, H: int, sigma: float, dst, stream=None):
    import torch

    _check("gs_blur", load().gs_blur(_ptr(src, torch.float32, "src"), C, W, H, sigma,
                                     _ptr(dst, torch.float32, "dst"), _stream(stream)))


def grad_stats(acc_xyz, acc_rgb, cnt, max_radius=None) -> GsGradStats:
    """The struct holds raw device pointers: the caller keeps the tensors alive."""
    import torch

    return GsGradStats(_ptr(acc_xyz, torch.float32, "acc_xyz"), _ptr(acc_rgb, torch.float32, "acc_rgb"),
                       _ptr(cnt, torch.int32, "cnt"), _ptr(max_radius, torch.int32, "max_radius"))


def gs_project_bwd_stats(P, n: int, sh_degree: int, cam: GsCamera, splats, act, n_active, grad2d, G, accumulate: bool,
                         sets, stream=None):
    """sets: list of up to two GsGradStats."""
    import torch

    arr = (GsGradStats * max(len(sets), 1))(*sets)
    _check("gs_project_bwd_stats", load().gs_project_bwd_stats(
        _ptr(P, torch.float32, "P"), n, sh_degree, ctypes.byref(cam), _ptr(splats, torch.float32, "splats"),
        _ptr(act, torch.int32, "act"), _ptr(n_active, torch.int32, "n_active"), _ptr(grad2d, torch.float32, "grad2d"),
        _ptr(G, torch.float32, "G"), int(bool(accumulate)), ctypes.cast(arr, ctypes.c_void_p), len(sets),
        _stream(stream)))


def gs_project_bwd_ex(P, n: int, sh_degree: int, opacity_act: int, cam: GsCamera, splats, act, n_active, grad2d, G,
                      accumulate: bool, sets, mask_loss: float = 0.0, stream=None):
    """gs_project_bwd_stats with the parameterisation chosen (GS_OPACITY_* | GS_VOLUME_MASK)."""
    import torch

    arr = (GsGradStats * max(len(sets), 1))(*sets)
    _check("gs_project_bwd_ex", load().gs_project_bwd_ex(
        _ptr(P, torch.float32, "P"), n, sh_degree, opacity_act, mask_loss, ctypes.byref(cam),
        _ptr(splats, torch.float32, "splats"), _ptr(act, torch.int32, "act"), _ptr(n_active, torch.int32, "n_active"),
        _ptr(grad2d, torch.float32, "grad2d"), _ptr(G, torch.float32, "G"), int(bool(accumulate)),
        ctypes.cast(arr, ctypes.c_void_p), len(sets), _stream(stream)))


class GsDensifyParams(ctypes.Structure):
    _fields_ = [("eps_xyz", ctypes.c_float), ("eps_rgb", ctypes.c_float), ("use_rgb", ctypes.c_int32),
                ("log_clone_max", ctypes.c_float), ("logit_min_opacity", ctypes.c_float),
                ("prune_big", ctypes.c_int32), ("max_screen_radius", ctypes.c_int32),
                ("log_max_world", ctypes.c_float), ("log_split_div", ctypes.c_float),
                ("mask_prune", ctypes.c_int32), ("mask_logit_min", ctypes.c_float),
                ("prune_mark", ctypes.c_void_p)]


def gs_densify_workspace_bytes(n: int) -> int:
    return int(load().gs_densify_workspace_bytes(n))


def gs_densify_plan(n: int, P, stats: GsGradStats, prm: GsDensifyParams, ws, counts, stream=None):
    """counts: int64 device tensor [4]."""
    import torch

    _check("gs_densify_plan", load().gs_densify_plan(
        n, _ptr(P, torch.float32, "P"), ctypes.byref(stats), ctypes.byref(prm), _ptr(ws, torch.uint8, "ws"),
        ws.numel(), _ptr(counts, torch.int64, "counts"), _stream(stream)))


class GsDensifyCarry(ctypes.Structure):
    _fields_ = [("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("row_bytes", ctypes.c_int32)]


def densify_carry(src, dst) -> GsDensifyCarry:
    """A per-Gaussian array (any dtype, rows of the same width) moved by gs_densify_apply. The struct
    holds raw device pointers: the caller keeps both tensors alive."""
    if not (src.is_cuda and dst.is_cuda and src.is_contiguous() and dst.is_contiguous() and src.dtype == dst.dtype):
        raise ValueError("carried arrays must be contiguous CUDA tensors of one dtype")
    row = src[0].numel() * src.element_size() if src.dim() > 1 else src.element_size()
    return GsDensifyCarry(src.data_ptr(), dst.data_ptr(), row)


def gs_densify_apply(n: int, P, m, v, frozen, carries, prm: GsDensifyParams, z, ws, capacity: int, P_out, m_out, v_out,
                     frozen_out, stream=None):
    """carries: list of GsDensifyCarry (at most 8)."""
    import torch

    arr = (GsDensifyCarry * max(len(carries), 1))(*carries)
    _check("gs_densify_apply", load().gs_densify_apply(
        n, _ptr(P, torch.float32, "P"), _ptr(m, torch.float32, "m"), _ptr(v, torch.float32, "v"),
        _ptr(frozen, torch.uint8, "frozen"), ctypes.cast(arr, ctypes.c_void_p), len(carries), ctypes.byref(prm),
        _ptr(z, torch.float32, "z"), _ptr(ws, torch.uint8, "ws"), ws.numel(), capacity,
        _ptr(P_out, torch.float32, "P_out"), _ptr(m_out, torch.float32, "m_out"), _ptr(v_out, torch.float32, "v_out"),
        _ptr(frozen_out, torch.uint8, "frozen_out"), _stream(stream)))


def gs_opacity_reset(n: int, P, m, v, logit_cap: float, frozen=None, stream=None):
    import torch

    _check("gs_opacity_reset", load().gs_opacity_reset(
        n, _ptr(P, torch.float32, "P"), _ptr(m, torch.float32, "m"), _ptr(v, torch.float32, "v"), logit_cap,
        _ptr(frozen, torch.uint8, "frozen"), _stream(stream)))


GS_MOMENTS_ZERO, GS_MOMENTS_RESCALE = 0, 1


def gs_opacity_to_abs(n: int, P, m, v, moments: int = GS_MOMENTS_ZERO, slope_sum=None, stream=None):
    import torch

    _check("gs_opacity_to_abs", load().gs_opacity_to_abs(n, _ptr(P, torch.float32, "P"), _ptr(m, torch.float32, "m"),
                                                         _ptr(v, torch.float32, "v"), moments,
                                                         _ptr(slope_sum, torch.float32, "slope_sum"),
                                                         _stream(stream)))


class GsRasterJob(ctypes.Structure):
    _fields_ = [("splats", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("ranges", ctypes.c_void_p),
                ("image", ctypes.c_void_p), ("t_final", ctypes.c_void_p), ("n_last", ctypes.c_void_p),
                ("dl_dimage", ctypes.c_void_p), ("frozen", ctypes.c_void_p), ("grad2d", ctypes.c_void_p),
                ("cam", GsCamera)]


def gs_render_fwd_batch(jobs_dev, n_jobs: int, width: int, height: int, tile: int, cfg, queue, stream=None):
    """jobs_dev: uint8 device tensor holding n_jobs GsRasterJob records."""
    import torch

    _check("gs_render_fwd_batch", load().gs_render_fwd_batch(
        _ptr(jobs_dev, torch.uint8, "jobs"), n_jobs, width, height, tile, None if cfg is None else ctypes.byref(cfg),
        _ptr(queue, torch.int32, "queue"), _stream(stream)))


def gs_raster_bwd_batch(jobs_dev, n_jobs: int, width: int, height: int, tile: int, cfg, queue, stream=None):
    import torch

    _check("gs_raster_bwd_batch", load().gs_raster_bwd_batch(
        _ptr(jobs_dev, torch.uint8, "jobs"), n_jobs, width, height, tile, None if cfg is None else ctypes.byref(cfg),
        _ptr(queue, torch.int32, "queue"), _stream(stream)))


def gs_render_bwd(P, n: int, sh_degree: int, cam: GsCamera, splats, vals, ranges, t_final, n_last, dl_dimage, frozen,
                  act, n_active, grad2d, G, acc_xyz=None, acc_rgb=None, cnt=None, stream=None):
    import torch

    _check("gs_render_bwd", load().gs_render_bwd(
        _ptr(P, torch.float32, "P"), n, sh_degree, ctypes.byref(cam), _ptr(splats, torch.float32, "splats"),
        _ptr(vals, torch.int32, "vals"), _ptr(ranges, torch.int32, "ranges"), _ptr(t_final, torch.float32, "t_final"),
        _ptr(n_last, torch.int32, "n_last"), _ptr(dl_dimage, torch.float32, "dl_dimage"),
        _ptr(frozen, torch.uint8, "frozen"), _ptr(act, torch.int32, "act"), _ptr(n_active, torch.int32, "n_active"),
        _ptr(grad2d, torch.float32, "grad2d"), _ptr(G, torch.float32, "G"), _ptr(acc_xyz, torch.float32, "acc_xyz"),
        _ptr(acc_rgb, torch.float32, "acc_rgb"), _ptr(cnt, torch.int32, "cnt"), _stream(stream)))


def gs_adam_masked_groups(P, G, m, v, n: int, act, n_active, lr, b1: float, b2: float, eps: float, step: int,
                          stream=None):
    """gs_adam_masked with len(lr) (6 or 7) group rates; the seventh is the volume-mask logit's."""
    import torch

    lra = (ctypes.c_float * len(lr))(*[float(x) for x in lr])
    _check("gs_adam_masked_groups", load().gs_adam_masked_groups(
        _ptr(P, torch.float32, "P"), _ptr(G, torch.float32, "G"), _ptr(m, torch.float32, "m"),
        _ptr(v, torch.float32, "v"), n, _ptr(act, torch.int32, "act"), _ptr(n_active, torch.int32, "n_active"), lra,
        len(lr), b1, b2, eps, step, _stream(stream)))


def gs_freeze_workspace_bytes(n: int) -> int:
    return int(load().gs_freeze_workspace_bytes(n))


def gs_freeze_update(n: int, acc_xyz, acc_rgb, cnt, frozen, eps_xyz: float, eps_rgb: float, mode: int, act, n_active,
                     ws, stream=None):
    import torch

    _check("gs_freeze_update", load().gs_freeze_update(
        n, _ptr(acc_xyz, torch.float32, "acc_xyz"), _ptr(acc_rgb, torch.float32, "acc_rgb"),
        _ptr(cnt, torch.int32, "cnt"), _ptr(frozen, torch.uint8, "frozen"), eps_xyz, eps_rgb, mode,
        _ptr(act, torch.int32, "act"), _ptr(n_active, torch.int32, "n_active"), _ptr(ws, torch.uint8, "ws"),
        ws.numel(), _stream(stream)))


def gs_freeze_update_noalloc(n: int, acc_xyz, acc_rgb, cnt, frozen, eps_xyz: float, eps_rgb: float, mode: int, act,
                             n_active, stream=None):
    """gs_freeze_update with the library's fixed scratch array instead of a workspace."""
    import torch

    _check("gs_freeze_update_noalloc", load().gs_freeze_update_noalloc(
        n, _ptr(acc_xyz, torch.float32, "acc_xyz"), _ptr(acc_rgb, torch.float32, "acc_rgb"),
        _ptr(cnt, torch.int32, "cnt"), _ptr(frozen, torch.uint8, "frozen"), eps_xyz, eps_rgb, mode,
        _ptr(act, torch.int32, "act"), _ptr(n_active, torch.int32, "n_active"), _stream(stream)))


def gs_adam_masked(P, G, m, v, n: int, act, n_active, lr, b1: float, b2: float, eps: float, step: int, stream=None):
    import torch

    lr6 = (ctypes.c_float * 6)(*[float(x) for x in lr])
    _check("gs_adam_masked", load().gs_adam_masked(
        _ptr(P, torch.float32, "P"), _ptr(G, torch.float32, "G"), _ptr(m, torch.float32, "m"),
        _ptr(v, torch.float32, "v"), n, _ptr(act, torch.int32, "act"), _ptr(n_active, torch.int32, "n_active"),
        lr6, b1, b2, eps, step, _stream(stream)))


def gs_adam_masked_devstep(P, G, m, v, n: int, act, n_active, lr_dev, b1: float, b2: float, eps: float, step_dev,
                           scratch, stream=None):
    """lr_dev: float32 device tensor of the six group rates."""
    import torch

    _check("gs_adam_masked_devstep", load().gs_adam_masked_devstep(
        _ptr(P, torch.float32, "P"), _ptr(G, torch.float32, "G"), _ptr(m, torch.float32, "m"),
        _ptr(v, torch.float32, "v"), n, _ptr(act, torch.int32, "act"), _ptr(n_active, torch.int32, "n_active"),
        _ptr(lr_dev, torch.float32, "lr_dev"), b1, b2, eps, _ptr(step_dev, torch.int64, "step"),
        _ptr(scratch, torch.float32, "scratch"), _stream(stream)))


MLP_PARAMS, MLP_WEIGHTS = 5313, 5184


def gs_pred_history(n: int, acc_xyz, acc_rgb, cnt, frozen, state, stream=None):
    import torch

    _check("gs_pred_history", load().gs_pred_history(
        n, _ptr(acc_xyz, torch.float32, "acc_xyz"), _ptr(acc_rgb, torch.float32, "acc_rgb"),
        _ptr(cnt, torch.int32, "cnt"), _ptr(frozen, torch.uint8, "frozen"), _ptr(state, torch.float32, "state"),
        _stream(stream)))


def gs_pred_features(n: int, P, acc_xyz, acc_rgb, cnt, state, k: int, K: int, eps_xyz: float, eps_rgb: float, X,
                     stream=None):
    import torch

    _check("gs_pred_features", load().gs_pred_features(
        n, _ptr(P, torch.float32, "P"), _ptr(acc_xyz, torch.float32, "acc_xyz"), _ptr(acc_rgb, torch.float32, "acc_rgb"),
        _ptr(cnt, torch.int32, "cnt"), _ptr(state, torch.float32, "state"), k, K, eps_xyz, eps_rgb,
        _ptr(X, torch.bfloat16, "X"), _stream(stream)))


def gs_mlp_fwd(n: int, X, wb, params, p, stream=None):
    import torch

    _check("gs_mlp_fwd", load().gs_mlp_fwd(n, _ptr(X, torch.bfloat16, "X"), _ptr(wb, torch.bfloat16, "wb"),
                                           _ptr(params, torch.float32, "params"), _ptr(p, torch.float32, "p"),
                                           _stream(stream)))


def gs_mlp_grad(n: int, X, y, w, inv_wsum: float, wb, params, grad, loss=None, stream=None):
    import torch

    _check("gs_mlp_grad", load().gs_mlp_grad(
        n, _ptr(X, torch.bfloat16, "X"), _ptr(y, torch.float32, "y"), _ptr(w, torch.float32, "w"), inv_wsum,
        _ptr(wb, torch.bfloat16, "wb"), _ptr(params, torch.float32, "params"), _ptr(grad, torch.float32, "grad"),
        _ptr(loss, torch.float32, "loss"), _stream(stream)))


def gs_mlp_adam(params, grad, m, v, wb, lr: float, b1: float, b2: float, eps: float, step: int, stream=None):
    import torch

    _check("gs_mlp_adam", load().gs_mlp_adam(
        _ptr(params, torch.float32, "params"), _ptr(grad, torch.float32, "grad"), _ptr(m, torch.float32, "m"),
        _ptr(v, torch.float32, "v"), _ptr(wb, torch.bfloat16, "wb"), lr, b1, b2, eps, step, _stream(stream)))


def gs_mlp_refresh(params, wb, stream=None):
    import torch

    _check("gs_mlp_refresh", load().gs_mlp_refresh(_ptr(params, torch.float32, "params"),
                                                   _ptr(wb, torch.bfloat16, "wb"), _stream(stream)))


def gs_freeze_apply(n: int, prob, tau: float, frozen, act, n_active, ws, stream=None):
    import torch

    _check("gs_freeze_apply", load().gs_freeze_apply(
        n, _ptr(prob, torch.float32, "prob"), tau, _ptr(frozen, torch.uint8, "frozen"), _ptr(act, torch.int32, "act"),
        _ptr(n_active, torch.int32, "n_active"), _ptr(ws, torch.uint8, "ws"), ws.numel(), _stream(stream)))


GS_FREEZE_RULE, GS_FREEZE_XYZ, GS_FREEZE_RANDOM, GS_FREEZE_MINGRAD = 0, 1, 2, 3


def gs_freeze_select_workspace_bytes(n: int) -> int:
    return int(load().gs_freeze_select_workspace_bytes(n))


def gs_freeze_select(n: int, acc_xyz, acc_rgb, cnt, frozen, eps_xyz: float, eps_rgb: float, strategy: int,
                     fraction: float, u, act, n_active, ws, stream=None):
    """Freeze update under an ablation strategy (GS_FREEZE_*); u: uniform draws [n] (RANDOM) or None."""
    import torch

    _check("gs_freeze_select", load().gs_freeze_select(
        n, _ptr(acc_xyz, torch.float32, "acc_xyz"), _ptr(acc_rgb, torch.float32, "acc_rgb"),
        _ptr(cnt, torch.int32, "cnt"), _ptr(frozen, torch.uint8, "frozen"), eps_xyz, eps_rgb, strategy, fraction,
        _ptr(u, torch.float32, "u"), _ptr(act, torch.int32, "act"), _ptr(n_active, torch.int32, "n_active"),
        _ptr(ws, torch.uint8, "ws"), ws.numel(), _stream(stream)))


def gs_psnr_workspace_bytes(S: int, H: int, W: int) -> int:
    return int(load().gs_psnr_workspace_bytes(S, H, W))


def gs_psnr(images, gts, S: int, H: int, W: int, ws, psnr, stream=None):
    import torch

    _check("gs_psnr", load().gs_psnr(_ptr(images, torch.float32, "images"), _ptr(gts, torch.float32, "gts"), S, H, W,
                                     _ptr(ws, torch.uint8, "ws"), ws.numel(), _ptr(psnr, torch.float32, "psnr"),
                                     _stream(stream)))


def gs_get_device_error(stream=None) -> int:
    """Synchronises the stream, returns and clears the device error bits."""
    flags = ctypes.c_uint32(0)
    st = load().gs_get_device_error(ctypes.byref(flags), _stream(stream))
    if st not in (0, 6):
        _check("gs_get_device_error", st)
    return int(flags.value)


def gs_status_string(status: int) -> str:
    return load().gs_status_string(status).decode()


def gs_raster_pair_counts(splats, vals, ranges, cam: GsCamera, n_last, frozen, counts, stream=None):
    """counts: int64 device tensor [3], added to (blended active, blended frozen, skipped)."""
    import torch

    _check("gs_raster_pair_counts", load().gs_raster_pair_counts(
        _ptr(splats, torch.float32, "splats"), _ptr(vals, torch.int32, "vals"), _ptr(ranges, torch.int32, "ranges"),
        ctypes.byref(cam), _ptr(n_last, torch.int32, "n_last"), _ptr(frozen, torch.uint8, "frozen"),
        _ptr(counts, torch.int64, "counts"), _stream(stream)))


def gs_launch_count() -> int:
    return int(load().gs_launch_count())


def gs_version() -> int:
    return int(load().gs_version())
