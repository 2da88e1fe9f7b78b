"""torch.autograd.Function wrappers of the rasterizer.

``render(r, means, log_scales, quats, opacity_logits, rgb, cams, xi=None)`` renders K views
(gs_project -> gs_bin_sort -> gs_raster_fwd) and returns (rgb [K,3,H,W], depth [K,H,W],
T_final [K,H,W]); its backward runs gs_raster_bwd -> gs_project_bwd on the same workspace.
The forward saves the per-pixel final transmittance and last-contributor index, so the
backward recomputes every alpha rather than storing it.

The camera pose enters through ``xi`` [K,6]: a left perturbation T <- Exp(xi) T of each view's
pose, evaluated at xi = 0 (the tensor must be zero; it exists so that its gradient is the
se(3) pose gradient (rho, phi), translation first). ``render_pose(r, g, cams, xi)`` is the
pose-only form used by tracking: the Gaussians are constants and only xi gets a gradient.

The backward reads the workspace state of its own forward (projected records, sorted pairs,
the record bit mask), so a Rasterizer holds one forward at a time: a second render on the
same Rasterizer before the first one's backward makes that backward raise.
"""
from __future__ import annotations

import weakref

import torch

from . import api


# xi tensors already found zero, by data_ptr: (weak reference, version counter). A tensor is read
# back to the host once, not on every render, so a render costs no device -> host synchronisation
# and can be captured in a CUDA graph once its xi has been validated
_xi_checked = {}


def _check_xi(xi, K, device):
    if xi is None:
        return torch.zeros((K, 6), device=device)
    if xi.shape != (K, 6):
        raise ValueError(f"xi must be [K, 6] = [{K}, 6], got {tuple(xi.shape)}")
    seen = _xi_checked.get(xi.data_ptr())
    if seen is not None and seen[0]() is xi and seen[1] == xi._version:
        return xi
    if torch.cuda.is_current_stream_capturing():
        raise RuntimeError("xi must be validated (rendered once) before a CUDA graph capture")
    if torch.count_nonzero(xi.detach()).item():
        raise ValueError("xi is the se(3) perturbation at which the pose gradient is taken: it must be zero")
    if len(_xi_checked) > 1024:
        _xi_checked.clear()
    _xi_checked[xi.data_ptr()] = (weakref.ref(xi), xi._version)
    return xi


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, r, pose_only, means, log_scales, quats, opacity_logits, rgb, xi, cams):
        g = api.Gaussians(means.detach(), log_scales.detach(), quats.detach(), opacity_logits.detach(),
                          rgb.detach())
        out = r.render(g, cams)
        r._autograd_version = getattr(r, "_autograd_version", 0) + 1
        ctx.version = r._autograd_version
        ctx.r, ctx.g, ctx.pose_only = r, g, pose_only
        ctx.save_for_backward(cams, out["rgb"], out["depth"], out["T"], out["last"])
        return out["rgb"], out["depth"], out["T"]

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_T):
        r = ctx.r
        if getattr(r, "_autograd_version", None) != ctx.version:
            raise RuntimeError("the Rasterizer rendered again before this backward: its workspace no longer holds "
                               "this forward's state")
        cams, rgb, depth, T, last = ctx.saved_tensors
        z = lambda t, ref: torch.zeros_like(ref) if t is None else t.contiguous()  # noqa: E731
        g_rgb, g_depth = z(g_rgb, rgb), z(g_depth, depth)
        g_T = None if g_T is None else g_T.contiguous()
        api.gs_raster_bwd(r.cfg, r.ws, rgb, depth, T, last, g_rgb, g_depth, g_T)
        d, N, K = rgb.device, r.N, r.K
        pose = torch.empty((K, 6), device=d)
        if ctx.pose_only:
            api.gs_project_bwd(r.cfg, ctx.g, cams, r.ws, {"pose": pose}, overwrite=True)
            return None, None, None, None, None, None, None, pose, None
        grads = {"means": torch.empty((N, 3), device=d), "log_scales": torch.empty((N, 3), device=d),
                 "quats": torch.empty((N, 4), device=d), "opacity_logits": torch.empty(N, device=d),
                 "rgb": torch.empty(r.color_shape(), device=d), "pose": pose}
        api.gs_project_bwd(r.cfg, ctx.g, cams, r.ws, grads, overwrite=True)
        cast = lambda t, like: t.to(like.dtype) if like.dtype != t.dtype else t  # noqa: E731
        g = ctx.g
        return (None, None, cast(grads["means"], g.means), cast(grads["log_scales"], g.log_scales),
                cast(grads["quats"], g.quats), cast(grads["opacity_logits"], g.opacity_logits),
                cast(grads["rgb"], g.rgb), pose, None)


def render(r: "api.Rasterizer", means, log_scales, quats, opacity_logits, rgb, cams, xi=None):
    """Differentiable render of K views; returns (rgb, depth, T_final)."""
    xi = _check_xi(xi, r.K, means.device)
    return _Render.apply(r, False, means, log_scales, quats, opacity_logits, rgb, xi, cams)


def render_pose(r: "api.Rasterizer", g: "api.Gaussians", cams, xi):
    """Pose-only differentiable render (the Gaussians are constants); returns (rgb, depth, T_final)."""
    xi = _check_xi(xi, r.K, cams.device)
    return _Render.apply(r, True, g.means, g.log_scales, g.quats, g.opacity_logits, g.rgb, xi, cams)
