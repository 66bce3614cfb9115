"""FP64 CPU oracle for the GSta training step.

TEST INFRASTRUCTURE ONLY: the test-suite, the package smoke check and the
benchmark's CPU-baseline leg are the only callers. The CUDA product never
imports this package, and this package imports nothing from the product.

The arithmetic lives in ``gsta_oracle.c`` (plain loops in double precision);
this module compiles it with gcc on first use and wraps each function for
numpy arrays. ``controller.py`` holds the host-side schedule of the method
(Eq. 5 thresholds, Eq. 7 early stop, plateau learning rate).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gsta_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

N_PARAMS = 59


def _plant() -> int:
    """Planted-mistake number of this process (environment GSTA_ORACLE_PLANT),
    0 -- the oracle itself -- unless the pins' own test set it."""
    return int(os.environ.get("GSTA_ORACLE_PLANT", "0") or 0)


def planted(k: int) -> bool:
    """Whether this process runs the copy of the oracle with planted mistake k
    (the Python modules' steps marked ``planted(k)``); False unless the pins'
    own test set GSTA_ORACLE_PLANT."""
    return _plant() == k


def build(force: bool = False, plant: int | None = None) -> str:
    """Compile the oracle with gcc (IEEE arithmetic: no fast-math, no FMA contraction).
    plant k >= 1 compiles the copy with planted mistake k, into the temporary
    directory (see PLANTED in gsta_oracle.c)."""
    plant = _plant() if plant is None else int(plant)
    out = _LIB
    if plant:
        import tempfile

        out = os.path.join(tempfile.gettempdir(), f"gsta_liboracle_plant{plant}_{os.getuid()}.so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
             f"-DORACLE_PLANT={plant}", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


class Cam(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("tile", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
        ("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3), ("campos", ctypes.c_double * 3),
        ("znear", ctypes.c_double), ("dilation", ctypes.c_double), ("bg", ctypes.c_double * 3),
    ]


def make_cam(cam, tile: int = 16, znear: float = 0.2, dilation: float = 0.3, bg=(0.0, 0.0, 0.0)) -> Cam:
    """Oracle camera from a ``synth.Camera``-like object (duck-typed)."""
    c = Cam()
    c.width, c.height, c.tile = int(cam.width), int(cam.height), int(tile)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.R[:] = [float(v) for v in np.asarray(cam.R, np.float64).reshape(9)]
    c.t[:] = [float(v) for v in np.asarray(cam.t, np.float64).reshape(3)]
    c.campos[:] = [float(v) for v in np.asarray(cam.campos, np.float64).reshape(3)]
    c.znear, c.dilation = float(znear), float(dilation)
    c.bg[:] = [float(v) for v in bg]
    return c


_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int32)
_up = ctypes.POINTER(ctypes.c_uint32)
_bp = ctypes.POINTER(ctypes.c_uint8)
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.or_sh_basis.argtypes = [_dp, _dp]
            L.or_sh_basis_grad.argtypes = [_dp, _dp]
            L.or_project_act.argtypes = [_i64, _dp, ctypes.POINTER(Cam), _i32, _i32, _i32, _dp, _dp, _dp, _dp, _dp,
                                         _dp, _ip, _ip, _dp]
            L.or_set_threads.argtypes = [_i32]
            L.or_max_threads.restype = _i32
            L.or_sort.argtypes = [_i64, _fp, _fp, _fp, _ip, _fp, _i32, _i32, _i32, _i32, _i64, _up, _up]
            L.or_sort.restype = _i64
            L.or_render.argtypes = [_i32, _i32, _i32, _dp, _i32, _dp, _dp, _dp, _dp, _up, _up, _dp, _dp, _ip, _dp]
            L.or_pixel_trace.argtypes = [_i32, _i32, _i32, _i32, _dp, _dp, _dp, _up, _up, _i32, _ip, _dp, _dp]
            L.or_pixel_trace.restype = _i32
            L.or_render_brute.argtypes = [_i64, _i32, _i32, _i32, _dp, _dp, _dp, _dp, _dp, _ip, _ip, _fp, _dp]
            L.or_loss.argtypes = [_i32, _i32, _dp, _dp, ctypes.c_double, _dp]
            L.or_loss.restype = ctypes.c_double
            L.or_loss_window.argtypes = [_i32, _i32, _dp, _dp, ctypes.c_double, _i32, _i32, _i32, _i32]
            L.or_loss_window.restype = ctypes.c_double
            L.or_render_bwd.argtypes = [_i64, _i32, _i32, _i32, _dp, _i32, _dp, _dp, _dp, _dp, _up, _up, _dp, _bp,
                                        _bp, _bp, _dp, _dp, _dp, _dp, _bp, _dp]
            L.or_render_pixels.argtypes = [_i64, _ip, _ip, _i32, _i32, _dp, _dp, _dp, _dp, _dp, _up, _up, _dp, _dp,
                                           _ip, _dp]
            L.or_render_pixels_locked.argtypes = [_i64, _ip, _ip, _i32, _i32, _dp, _dp, _dp, _dp, _dp, _up, _up,
                                                  _i32, _i64, _bp, _dp]
            L.or_project_bwd_act.argtypes = [_i64, _dp, ctypes.POINTER(Cam), _i32, _i32, _i32, _dp, ctypes.c_double,
                                             _bp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
            L.or_adam.argtypes = [_i64, _dp, _dp, _dp, _dp, _bp, _dp, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, _i64]
            L.or_freeze_update.argtypes = [_i64, _fp, _fp, _ip, _bp, ctypes.c_float, ctypes.c_float, _i32, _ip]
            L.or_freeze_update.restype = _i64
            L.or_psnr.argtypes = [_i32, _i32, _i32, _dp, _dp, _dp]
            L.or_mlp_nparams.restype = _i32
            L.or_freeze_apply.argtypes = [_i64, _fp, ctypes.c_float, _bp, _ip]
            L.or_freeze_apply.restype = _i64
            L.or_bf16.argtypes = [ctypes.c_double]
            L.or_bf16.restype = ctypes.c_double
            L.or_pred_history.argtypes = [_i64, _fp, _fp, _ip, _bp, _dp]
            L.or_pred_features.argtypes = [_i64, _dp, _fp, _fp, _ip, _dp, _i32, _i32, ctypes.c_double,
                                           ctypes.c_double, _dp]
            L.or_mlp_forward.argtypes = [_i64, _dp, _dp, _i32, _dp]
            L.or_mlp_loss_grad.argtypes = [_i64, _dp, _dp, _dp, _dp, _i32, _dp, _dp]
            L.or_mlp_loss_grad.restype = ctypes.c_double
            L.or_mlp_adam.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, _i64]
            _lib = L
    return _lib


def _p(a, t):
    return None if a is None else a.ctypes.data_as(t)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def set_threads(n: int):
    """Host threads of the oracle's parallel loops (results do not depend on it)."""
    lib().or_set_threads(int(n))


def max_threads() -> int:
    return int(lib().or_max_threads())


def sh_basis(d) -> np.ndarray:
    d = _c(d, np.float64)
    out = np.zeros(16)
    lib().or_sh_basis(_p(d, _dp), _p(out, _dp))
    return out


def sh_basis_grad(d) -> np.ndarray:
    d = _c(d, np.float64)
    out = np.zeros((16, 3))
    lib().or_sh_basis_grad(_p(d, _dp), _p(out, _dp))
    return out


def project(params, cam: Cam, sh_degree: int = 3, smooth: bool = False, opacity_act: int = 0, mask=None) -> dict:
    """Per-Gaussian projection (Eq. 1) and SH colour; opacity_act 1: opacity = |x|
    (the finetuning stage's activation, Sec. 4.1) instead of sigmoid(x); mask:
    volume-mask logits [n] (Sec. 3.3), a Gaussian whose hard mask is 0 culled."""
    P = _c(params, np.float64)
    mk = None if mask is None else _c(mask, np.float64)
    n = P.shape[0]
    out = dict(mean2d=np.zeros((n, 2)), conic=np.zeros((n, 3)), depth=np.zeros(n), opacity=np.zeros(n),
               rgb=np.zeros((n, 3)), radius=np.zeros(n, np.int32), rect=np.zeros((n, 4), np.int32),
               margin=np.zeros(n))
    lib().or_project_act(n, _p(P, _dp), ctypes.byref(cam), sh_degree, int(smooth), int(opacity_act), _p(mk, _dp),
                         _p(out["mean2d"], _dp),
                     _p(out["conic"], _dp), _p(out["depth"], _dp), _p(out["opacity"], _dp), _p(out["rgb"], _dp),
                     _p(out["radius"], _ip), _p(out["rect"], _ip), _p(out["margin"], _dp))
    r = out["rect"]
    out["tiles_touched"] = ((r[:, 2] - r[:, 0]) * (r[:, 3] - r[:, 1])).astype(np.int32)
    return out


def sort(mean2d_f32, conic_f32, opacity_f32, radius, depth_f32, W: int, H: int, tile: int = 16,
         smooth: bool = False, capacity: int | None = None):
    """Tile/depth order of single-precision splats (mean2d [n][2], conic [n][3],
    opacity [n], radius [n], depth [n]). Returns (vals uint32[P], ranges
    uint32[tiles, 2])."""
    m = _c(mean2d_f32, np.float32)
    q = _c(conic_f32, np.float32)
    o = _c(opacity_f32, np.float32)
    r = _c(radius, np.int32)
    d = _c(depth_f32, np.float32)
    n = r.shape[0]
    tiles = ((W + tile - 1) // tile) * ((H + tile - 1) // tile)
    args = (_p(m, _fp), _p(q, _fp), _p(o, _fp), _p(r, _ip), _p(d, _fp), W, H, tile, int(smooth))
    if capacity is None:
        capacity = abs(lib().or_sort(n, *args, 0, None, None))
    vals = np.zeros(max(capacity, 1), np.uint32)
    ranges = np.zeros((tiles, 2), np.uint32)
    P = lib().or_sort(n, *args, capacity, _p(vals, _up), _p(ranges, _up))
    if P < 0:
        raise OverflowError(f"sort needs {-P} entries, capacity {capacity}")
    return vals[:P], ranges


def sort_proj(proj: dict, W: int, H: int, tile: int = 16, smooth: bool = False, capacity: int | None = None):
    """sort() of a projection's values rounded to single precision."""
    return sort(proj["mean2d"].astype(np.float32), proj["conic"].astype(np.float32),
                proj["opacity"].astype(np.float32), proj["radius"], proj["depth"].astype(np.float32), W, H, tile,
                smooth, capacity)


def sort_records(rec, W: int, H: int, tile: int = 16, capacity: int | None = None):
    """sort() of float32 splat records [n][12] (the C-ABI layout: mean 0-1,
    conic 2-4, opacity 5, depth 9, radius bits 10)."""
    rec = np.ascontiguousarray(rec, np.float32)
    return sort(rec[:, 0:2], rec[:, 2:5], rec[:, 5], rec[:, 10].view(np.int32), rec[:, 9], W, H, tile,
                capacity=capacity)


def render(proj: dict, vals, ranges, cam: Cam, smooth: bool = False) -> dict:
    """Tiled compositing (Eq. 2)."""
    W, H = cam.width, cam.height
    bg = np.array(list(cam.bg), np.float64)
    image = np.zeros((3, H, W))
    tfin = np.zeros((H, W))
    nlast = np.zeros((H, W), np.int32)
    margin = np.zeros((H, W))
    lib().or_render(W, H, cam.tile, _p(bg, _dp), int(smooth), _p(_c(proj["mean2d"], np.float64), _dp),
                    _p(_c(proj["conic"], np.float64), _dp), _p(_c(proj["opacity"], np.float64), _dp),
                    _p(_c(proj["rgb"], np.float64), _dp), _p(_c(vals, np.uint32), _up),
                    _p(_c(ranges, np.uint32), _up), _p(image, _dp), _p(tfin, _dp), _p(nlast, _ip), _p(margin, _dp))
    return dict(image=image, t_final=tfin, n_last=nlast, margin=margin)


def pixel_trace(proj: dict, vals, ranges, cam: Cam, px: int, py: int, cap: int = 100000):
    """(list positions, alphas, transmittance in front) of one pixel's contributors."""
    pos = np.zeros(cap, np.int32)
    al = np.zeros(cap)
    tr = np.zeros(cap)
    k = lib().or_pixel_trace(px, py, cam.width, cam.tile, _p(_c(proj["mean2d"], np.float64), _dp),
                             _p(_c(proj["conic"], np.float64), _dp), _p(_c(proj["opacity"], np.float64), _dp),
                             _p(_c(vals, np.uint32), _up), _p(_c(ranges, np.uint32), _up), cap, _p(pos, _ip),
                             _p(al, _dp), _p(tr, _dp))
    return pos[:k], al[:k], tr[:k]


def render_brute(proj: dict, cam: Cam) -> np.ndarray:
    W, H = cam.width, cam.height
    bg = np.array(list(cam.bg), np.float64)
    n = proj["radius"].shape[0]
    image = np.zeros((3, H, W))
    lib().or_render_brute(n, W, H, cam.tile, _p(bg, _dp), _p(_c(proj["mean2d"], np.float64), _dp),
                          _p(_c(proj["conic"], np.float64), _dp), _p(_c(proj["opacity"], np.float64), _dp),
                          _p(_c(proj["rgb"], np.float64), _dp), _p(_c(proj["radius"], np.int32), _ip),
                          _p(_c(proj["rect"], np.int32), _ip), _p(_c(proj["depth"], np.float32), _fp),
                          _p(image, _dp))
    return image


def loss(image, gt, lam: float = 0.2, grad: bool = True):
    """Eq. 3. Returns (loss, dL/dimage or None)."""
    x = _c(image, np.float64)
    y = _c(gt, np.float64)
    H, W = x.shape[1], x.shape[2]
    g = np.zeros_like(x) if grad else None
    val = lib().or_loss(H, W, _p(x, _dp), _p(y, _dp), lam, _p(g, _dp))
    return val, g


def loss_window(image, gt, x0: int, y0: int, x1: int, y1: int, lam: float = 0.2) -> float:
    """The window [x0, x1) x [y0, y1)'s share of Eq. 3 (see or_loss_window)."""
    x = _c(image, np.float64)
    y = _c(gt, np.float64)
    H, W = x.shape[1], x.shape[2]
    return lib().or_loss_window(H, W, _p(x, _dp), _p(y, _dp), lam, x0, y0, x1, y1)


def render_pixels_locked(proj: dict, vals, ranges, cam: Cam, px, py, dec=None):
    """or_render_pixels_locked: with dec None, renders and records the
    decisions (returns image, dec); with dec given, replays them."""
    px = _c(px, np.int32)
    py = _c(py, np.int32)
    k = px.shape[0]
    r = _c(ranges, np.uint32).reshape(-1, 2)
    stride = int(max(1, (r[:, 1] - r[:, 0]).max()))
    mode = 0 if dec is None else 1
    if dec is None:
        dec = np.zeros((k, stride), np.uint8)
    bg = np.array(list(cam.bg), np.float64)
    image = np.zeros((3, k))
    lib().or_render_pixels_locked(k, _p(px, _ip), _p(py, _ip), cam.width, cam.tile, _p(bg, _dp),
                                  _p(_c(proj["mean2d"], np.float64), _dp), _p(_c(proj["conic"], np.float64), _dp),
                                  _p(_c(proj["opacity"], np.float64), _dp), _p(_c(proj["rgb"], np.float64), _dp),
                                  _p(_c(vals, np.uint32), _up), _p(r, _up), mode, stride, _p(dec, _bp),
                                  _p(image, _dp))
    return image, dec


def render_pixels(proj: dict, vals, ranges, cam: Cam, px, py) -> dict:
    """Eq. 2 at the listed pixels only."""
    px = _c(px, np.int32)
    py = _c(py, np.int32)
    k = px.shape[0]
    bg = np.array(list(cam.bg), np.float64)
    out = dict(image=np.zeros((3, k)), t_final=np.zeros(k), n_last=np.zeros(k, np.int32), margin=np.zeros(k))
    lib().or_render_pixels(k, _p(px, _ip), _p(py, _ip), cam.width, cam.tile, _p(bg, _dp),
                           _p(_c(proj["mean2d"], np.float64), _dp), _p(_c(proj["conic"], np.float64), _dp),
                           _p(_c(proj["opacity"], np.float64), _dp), _p(_c(proj["rgb"], np.float64), _dp),
                           _p(_c(vals, np.uint32), _up), _p(_c(ranges, np.uint32), _up), _p(out["image"], _dp),
                           _p(out["t_final"], _dp), _p(out["n_last"], _ip), _p(out["margin"], _dp))
    return out


def render_bwd(proj: dict, vals, ranges, cam: Cam, dl_dimage, frozen=None, amb=None, smooth: bool = False,
               tile_mask=None) -> dict:
    W, H = cam.width, cam.height
    n = proj["opacity"].shape[0]
    bg = np.array(list(cam.bg), np.float64)
    out = dict(d_mean2d=np.zeros((n, 2)), d_conic=np.zeros((n, 3)), d_opacity=np.zeros(n), d_rgb=np.zeros((n, 3)),
               tainted=np.zeros(n, np.uint8), amb_abs=np.zeros((n, 9)))
    fr = None if frozen is None else _c(frozen, np.uint8)
    am = None if amb is None else _c(amb, np.uint8)
    tm = None if tile_mask is None else _c(tile_mask, np.uint8)
    lib().or_render_bwd(n, W, H, cam.tile, _p(bg, _dp), int(smooth), _p(_c(proj["mean2d"], np.float64), _dp),
                        _p(_c(proj["conic"], np.float64), _dp), _p(_c(proj["opacity"], np.float64), _dp),
                        _p(_c(proj["rgb"], np.float64), _dp), _p(_c(vals, np.uint32), _up),
                        _p(_c(ranges, np.uint32), _up), _p(_c(dl_dimage, np.float64), _dp), _p(fr, _bp),
                        _p(am, _bp), _p(tm, _bp), _p(out["d_mean2d"], _dp), _p(out["d_conic"], _dp), _p(out["d_opacity"], _dp),
                        _p(out["d_rgb"], _dp), _p(out["tainted"], _bp), _p(out["amb_abs"], _dp))
    return out


def project_bwd(params, cam: Cam, grads2d: dict, frozen=None, sh_degree: int = 3, smooth: bool = False,
                opacity_act: int = 0, mask=None, mask_loss: float = 0.0) -> dict:
    """Chain rule to the 59 parameters (G), freeze statistics, and with volume
    masks the straight-through gradient of each mask logit (G_mask)."""
    P = _c(params, np.float64)
    n = P.shape[0]
    G = np.zeros((n, N_PARAMS))
    xn = np.zeros(n)
    rn = np.zeros(n)
    fr = None if frozen is None else _c(frozen, np.uint8)
    mk = None if mask is None else _c(mask, np.float64)
    gm = np.zeros(n)
    lib().or_project_bwd_act(n, _p(P, _dp), ctypes.byref(cam), sh_degree, int(smooth), int(opacity_act), _p(mk, _dp),
                             float(mask_loss), _p(fr, _bp),
                             _p(_c(grads2d["d_mean2d"], np.float64), _dp), _p(_c(grads2d["d_conic"], np.float64), _dp),
                             _p(_c(grads2d["d_opacity"], np.float64), _dp), _p(_c(grads2d["d_rgb"], np.float64), _dp),
                             _p(G, _dp), _p(gm, _dp), _p(xn, _dp), _p(rn, _dp))
    return dict(G=G, G_mask=gm, xyz_norm=xn, rgb_norm=rn)


def adam(P, G, M, V, frozen, lr, step: int, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-15):
    """In-place masked Adam on float64 (n, 59) arrays."""
    for a in (P, M, V):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lr = _c(lr, np.float64)
    fr = None if frozen is None else _c(frozen, np.uint8)
    lib().or_adam(P.shape[0], _p(P, _dp), _p(_c(G, np.float64), _dp), _p(M, _dp), _p(V, _dp), _p(fr, _bp),
                  _p(lr, _dp), b1, b2, eps, step)


def freeze_update(acc_xyz, acc_rgb, cnt, frozen, eps_xyz: float, eps_rgb: float, mode: int):
    """In-place on float32 acc arrays, int32 cnt and uint8 frozen. Returns act (int32, ascending)."""
    for a, dt in ((acc_xyz, np.float32), (acc_rgb, np.float32), (cnt, np.int32), (frozen, np.uint8)):
        assert a.dtype == dt and a.flags.c_contiguous
    n = frozen.shape[0]
    act = np.zeros(max(n, 1), np.int32)
    k = lib().or_freeze_update(n, _p(acc_xyz, _fp), _p(acc_rgb, _fp), _p(cnt, _ip), _p(frozen, _bp),
                               np.float32(eps_xyz), np.float32(eps_rgb), mode, _p(act, _ip))
    return act[:k]


def psnr(images, gts) -> np.ndarray:
    x = _c(images, np.float64)
    y = _c(gts, np.float64)
    S, H, W = x.shape[0], x.shape[2], x.shape[3]
    out = np.zeros(S)
    lib().or_psnr(S, H, W, _p(x, _dp), _p(y, _dp), _p(out, _dp))
    return out


# ---------------------------------------------------------------------------
# Whole-step compositions (each stage above, in the paper's order).
# ---------------------------------------------------------------------------

def forward(params, cam: Cam, sh_degree: int = 3, smooth: bool = False, opacity_act: int = 0) -> dict:
    """Projection, per-tile depth order and compositing for one view."""
    proj = project(params, cam, sh_degree, smooth, opacity_act)
    vals, ranges = sort_proj(proj, cam.width, cam.height, cam.tile, smooth)
    ren = render(proj, vals, ranges, cam, smooth)
    return dict(proj=proj, vals=vals, ranges=ranges, **ren)


def loss_and_grad(params, cam: Cam, gt, frozen=None, sh_degree: int = 3, smooth: bool = False,
                  lam: float = 0.2, opacity_act: int = 0) -> dict:
    """Forward, Eq. 3 loss and the analytic gradient of the loss w.r.t. all 59 parameters."""
    f = forward(params, cam, sh_degree, smooth, opacity_act)
    L, dimg = loss(f["image"], gt, lam)
    g2 = render_bwd(f["proj"], f["vals"], f["ranges"], cam, dimg, frozen, smooth=smooth)
    pb = project_bwd(params, cam, g2, frozen, sh_degree, smooth, opacity_act)
    return dict(loss=L, dl_dimage=dimg, grads2d=g2, **pb, fwd=f)


def loss_only(params, cam: Cam, gt, sh_degree: int = 3, smooth: bool = False, lam: float = 0.2,
              opacity_act: int = 0) -> float:
    f = forward(params, cam, sh_degree, smooth, opacity_act)
    return loss(f["image"], gt, lam, grad=False)[0]


# ---------------------------------------------------------------------------
# Learned freeze predictor (not in the paper; the reference for its kernels).
# ---------------------------------------------------------------------------
MLP_IN, MLP_H = 16, 64
MLP_OFF = dict(W1=0, b1=1024, W2=1088, b2=5184, W3=5248, b3=5312)


def mlp_nparams() -> int:
    return int(lib().or_mlp_nparams())


def bf16(x) -> np.ndarray:
    """Round-to-nearest-even bfloat16 of float32(x), element-wise."""
    f = np.asarray(x, np.float32).copy()
    b = f.view(np.uint32)
    b += np.uint32(0x7FFF) + ((b >> 16) & np.uint32(1))
    b &= np.uint32(0xFFFF0000)
    return b.view(np.float32).astype(np.float64)


def pred_history(acc_xyz, acc_rgb, cnt, frozen, state):
    """In-place update of the [n][12] float64 predictor state at a statistics boundary."""
    assert state.dtype == np.float64 and state.flags.c_contiguous
    fr = None if frozen is None else _c(frozen, np.uint8)
    lib().or_pred_history(state.shape[0], _p(_c(acc_xyz, np.float32), _fp), _p(_c(acc_rgb, np.float32), _fp),
                          _p(_c(cnt, np.int32), _ip), _p(fr, _bp), _p(state, _dp))


def pred_features(P, acc_xyz, acc_rgb, cnt, state, k: int, K: int, eps_xyz: float, eps_rgb: float) -> np.ndarray:
    P = _c(P, np.float64)
    n = P.shape[0]
    X = np.zeros((n, MLP_IN))
    lib().or_pred_features(n, _p(P, _dp), _p(_c(acc_xyz, np.float32), _fp), _p(_c(acc_rgb, np.float32), _fp),
                           _p(_c(cnt, np.int32), _ip), _p(_c(state, np.float64), _dp), k, K, eps_xyz, eps_rgb,
                           _p(X, _dp))
    return X


def mlp_forward(X, prm, round_bf16: bool = True) -> np.ndarray:
    X = _c(X, np.float64)
    p = np.zeros(X.shape[0])
    lib().or_mlp_forward(X.shape[0], _p(X, _dp), _p(_c(prm, np.float64), _dp), int(round_bf16), _p(p, _dp))
    return p


def mlp_loss_grad(X, y, prm, w=None, round_bf16: bool = True, with_abs: bool = False):
    """(loss, gradient) or, with ``with_abs``, (loss, gradient, sum of |per-row terms|)."""
    X = _c(X, np.float64)
    g = np.zeros(mlp_nparams())
    a = np.zeros(mlp_nparams()) if with_abs else None
    wv = None if w is None else _c(w, np.float64)
    L = lib().or_mlp_loss_grad(X.shape[0], _p(X, _dp), _p(_c(y, np.float64), _dp), _p(wv, _dp),
                               _p(_c(prm, np.float64), _dp), int(round_bf16), _p(g, _dp), _p(a, _dp))
    return (L, g, a) if with_abs else (L, g)


def mlp_adam(prm, grad, m, v, lr: float, step: int, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    for a in (prm, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().or_mlp_adam(_p(prm, _dp), _p(_c(grad, np.float64), _dp), _p(m, _dp), _p(v, _dp), lr, b1, b2, eps, step)


def freeze_apply(prob, tau: float, frozen):
    """In-place frozen |= prob > tau (uint8 frozen); returns the active list."""
    assert frozen.dtype == np.uint8 and frozen.flags.c_contiguous
    n = frozen.shape[0]
    act = np.zeros(max(n, 1), np.int32)
    k = lib().or_freeze_apply(n, _p(_c(prob, np.float32), _fp), np.float32(tau), _p(frozen, _bp), _p(act, _ip))
    return act[:k]
