"""torch.autograd wrappers over the C ABI.

``rasterize(P, cam)`` renders the Gaussians (gs_project, gs_sort,
gs_render_fwd); its backward is the hand-written rasteriser and projection
backward (gs_raster_bwd, gs_project_bwd), which recomputes each pixel's
transmittance from the value the forward left over instead of storing
per-pixel lists. Gaussians marked in ``frozen`` receive no gradient (their
rows of the returned gradient are zero), as in Sec. 3.2.4.

``ssim_l1_loss(image, gt)`` is Eq. 3 (gs_loss) with its own backward.
Nothing here computes: it marshals tensors and calls the library.
"""
from __future__ import annotations

import torch

from . import lib


class RasterizeGaussians(torch.autograd.Function):
    @staticmethod
    def forward(ctx, P, cam, sh_degree=3, capacity=None, frozen=None):
        n = P.shape[0]
        dev = P.device
        P = P.contiguous()
        splats = torch.empty((n, lib.SPLAT), dtype=torch.float32, device=dev)
        lib.gs_project(P, n, sh_degree, cam, splats)
        if capacity is None:
            capacity = int(splats[:, 11].contiguous().view(torch.int32).to(torch.int64).sum().item()) + 1024
        ws = torch.empty(lib.gs_sort_workspace_bytes(n, capacity, cam), dtype=torch.uint8, device=dev)
        vals = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
        ranges = torch.empty((cam.tiles, 2), dtype=torch.int32, device=dev)
        count = torch.empty(1, dtype=torch.int64, device=dev)
        lib.gs_sort(splats, n, cam, ws, capacity, vals, ranges, count)
        H, W = cam.height, cam.width
        image = torch.empty((3, H, W), dtype=torch.float32, device=dev)
        t_final = torch.empty((H, W), dtype=torch.float32, device=dev)
        n_last = torch.empty((H, W), dtype=torch.int32, device=dev)
        lib.gs_render_fwd(splats, vals, ranges, cam, image, t_final, n_last)
        ctx.save_for_backward(P, splats, vals, ranges, t_final, n_last)
        ctx.cam, ctx.sh_degree, ctx.frozen = cam, sh_degree, frozen
        ctx.mark_non_differentiable(t_final, n_last)
        return image, t_final, n_last

    @staticmethod
    def backward(ctx, dl_dimage, _dt, _dn):
        P, splats, vals, ranges, t_final, n_last = ctx.saved_tensors
        n = P.shape[0]
        dev = P.device
        grad2d = torch.zeros((n, lib.GRAD2D), dtype=torch.float32, device=dev)
        G = torch.zeros((n, lib.ROW), dtype=torch.float32, device=dev)
        frozen = ctx.frozen
        if frozen is None:
            act = torch.arange(n, dtype=torch.int32, device=dev)
        else:
            act = torch.nonzero(frozen == 0).flatten().to(torch.int32)
        n_active = torch.tensor([act.numel()], dtype=torch.int32, device=dev)
        lib.gs_raster_bwd(splats, vals, ranges, ctx.cam, t_final, n_last, dl_dimage.contiguous(), frozen, grad2d)
        lib.gs_project_bwd(P, n, ctx.sh_degree, ctx.cam, splats, act, n_active, grad2d, G)
        return G, None, None, None, None


class SsimL1Loss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, image, gt, lam=0.2):
        H, W = image.shape[1], image.shape[2]
        ws = torch.empty(lib.gs_loss_workspace_bytes(H, W), dtype=torch.uint8, device=image.device)
        loss = torch.empty(1, dtype=torch.float32, device=image.device)
        dl = torch.empty_like(image)
        lib.gs_loss(image.contiguous(), gt.contiguous(), H, W, lam, ws, loss, dl)
        ctx.save_for_backward(dl)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (dl,) = ctx.saved_tensors
        return dl * g, None, None


def rasterize(P: torch.Tensor, cam: lib.GsCamera, sh_degree: int = 3, capacity: int | None = None,
              frozen: torch.Tensor | None = None) -> torch.Tensor:
    """Image [3, H, W] of the Gaussians P [N, 64]; differentiable in P."""
    return RasterizeGaussians.apply(P, cam, sh_degree, capacity, frozen)[0]


def ssim_l1_loss(image: torch.Tensor, gt: torch.Tensor, lam: float = 0.2) -> torch.Tensor:
    """Eq. 3: (1 - lam) L1 + lam (1 - SSIM); differentiable in image."""
    return SsimL1Loss.apply(image, gt, lam)
