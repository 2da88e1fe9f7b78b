"""Python face of the C ABI: one function per ``gs_*`` entry point, plus a small
``Rasterizer`` that owns a workspace and chains the calls of a forward render and
of its backward pass.

PyTorch only provides device memory and streams here. Every computation runs in
the sm_103a kernels of ``libgs.so``; if the library cannot be loaded the calls
raise instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import dataclasses

import torch

from . import _lib
from ._lib import GsAdam, GsConfig, GsGaussians, GsGrads, GsWsLayout, call

DTYPES = {torch.float32: _lib.GS_F32, torch.bfloat16: _lib.GS_BF16, torch.float16: _lib.GS_F16}
TILE = 16


def _p(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "tensors passed to the library must be contiguous CUDA tensors"
    return ctypes.c_void_p(t.data_ptr())


def _s(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


COLOR_RGB, COLOR_SH = 0, 1


def make_config(width, height, num_views, num_gaussians, pair_capacity, near_plane=0.2, lambda_depth=0.1,
                fwd_px=0, bwd_px=0, fwd_chunk=0, bwd_chunk=0, sh_degree=None, blocks_per_sm=0):
    """sh_degree None: the rgb array is the colour [N,3]; 0..3: it holds spherical-harmonic
    coefficients [N,(sh_degree+1)^2,3] evaluated per view."""
    mode = COLOR_RGB if sh_degree is None else COLOR_SH
    return GsConfig(int(width), int(height), TILE, int(num_views), int(num_gaussians), int(pair_capacity),
                    float(near_plane), float(lambda_depth), int(fwd_px), int(bwd_px), int(fwd_chunk), int(bwd_chunk),
                    mode, int(sh_degree or 0), int(blocks_per_sm))


def workspace_size(cfg: GsConfig) -> int:
    n = ctypes.c_size_t()
    call("gs_workspace_size", ctypes.byref(cfg), ctypes.byref(n))
    return n.value


def workspace_layout(cfg: GsConfig) -> GsWsLayout:
    out = GsWsLayout()
    call("gs_workspace_layout", ctypes.byref(cfg), ctypes.byref(out))
    return out


@dataclasses.dataclass
class Gaussians:
    """Device tensors of N Gaussians (see include/gs.h for layouts)."""
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logits: torch.Tensor
    rgb: torch.Tensor

    @property
    def N(self) -> int:
        return int(self.means.shape[0])

    def struct(self) -> GsGaussians:
        dt = DTYPES[self.log_scales.dtype]
        for t in (self.quats, self.opacity_logits, self.rgb):
            assert DTYPES[t.dtype] == dt, "log_scales, quats, opacity_logits and rgb share one storage dtype"
        return GsGaussians(_p(self.means), _p(self.log_scales), _p(self.quats), _p(self.opacity_logits), _p(self.rgb),
                           dt, DTYPES[self.means.dtype])

    @staticmethod
    def from_numpy(params, device="cuda", dtype=torch.float32, means_dtype=torch.float32) -> "Gaussians":
        means, ls, qs, lg, rgb = params
        t = lambda a, d: torch.as_tensor(a).to(device=device, dtype=d).contiguous()  # noqa: E731
        return Gaussians(t(means, means_dtype), t(ls, dtype), t(qs, dtype), t(lg, dtype), t(rgb, dtype))


def workspace(cfg: GsConfig, device="cuda") -> torch.Tensor:
    # torch's caching allocator returns blocks aligned to at least 512 bytes
    ws = torch.empty(workspace_size(cfg), dtype=torch.uint8, device=device)
    assert ws.data_ptr() % 256 == 0
    return ws


# ----------------------------------------------------------------------------- entry points

def gs_project(cfg, g: Gaussians, cams: torch.Tensor, ws: torch.Tensor, stream=None):
    gs = g.struct()
    call("gs_project", ctypes.byref(cfg), ctypes.byref(gs), _p(cams), _p(ws), ws.numel(), _s(stream))


def gs_bin_sort(cfg, ws, stream=None):
    call("gs_bin_sort", ctypes.byref(cfg), _p(ws), ws.numel(), _s(stream))


def gs_raster_fwd(cfg, ws, rgb, depth, T_final, last, stream=None):
    call("gs_raster_fwd", ctypes.byref(cfg), _p(ws), ws.numel(), _p(rgb), _p(depth), _p(T_final), _p(last),
         _s(stream))


def gs_raster_fwd_l1(cfg, ws, rgb, depth, T_final, last, rgb_target, depth_target, dL_drgb, dL_ddepth, loss,
                     stream=None):
    call("gs_raster_fwd_l1", ctypes.byref(cfg), _p(ws), ws.numel(), _p(rgb), _p(depth), _p(T_final), _p(last),
         _p(rgb_target), _p(depth_target), _p(dL_drgb), _p(dL_ddepth), _p(loss), _s(stream))


def gs_raster_fwd_l1_bwd(cfg, ws, rgb, depth, T_final, last, rgb_target, depth_target, dL_drgb, dL_ddepth, loss,
                         stream=None):
    """gs_raster_fwd_l1 followed by gs_raster_bwd (no dL/dT) in one launch."""
    call("gs_raster_fwd_l1_bwd", ctypes.byref(cfg), _p(ws), ws.numel(), _p(rgb), _p(depth), _p(T_final), _p(last),
         _p(rgb_target), _p(depth_target), _p(dL_drgb), _p(dL_ddepth), _p(loss), _s(stream))


def gs_raster_fwd_occluded(cfg, ws, rgb, depth, T_final, last, ext_depth, ext_rgb=None, stream=None):
    call("gs_raster_fwd_occluded", ctypes.byref(cfg), _p(ws), ws.numel(), _p(rgb), _p(depth), _p(T_final), _p(last),
         _p(ext_depth), _p(ext_rgb), _s(stream))


def gs_raster_fwd_stats(cfg, ws, rgb, depth, T_final, last, stream=None):
    call("gs_raster_fwd_stats", ctypes.byref(cfg), _p(ws), ws.numel(), _p(rgb), _p(depth), _p(T_final), _p(last),
         _s(stream))


def gs_loss_l1(cfg, rgb, depth, rgb_target, depth_target, dL_drgb, dL_ddepth, loss, ws, stream=None):
    call("gs_loss_l1", ctypes.byref(cfg), _p(rgb), _p(depth), _p(rgb_target), _p(depth_target), _p(dL_drgb),
         _p(dL_ddepth), _p(loss), _p(ws), ws.numel(), _s(stream))


def gs_raster_bwd(cfg, ws, rgb, depth, T_final, last, dL_drgb, dL_ddepth, dL_dT=None, stream=None):
    call("gs_raster_bwd", ctypes.byref(cfg), _p(ws), ws.numel(), _p(rgb), _p(depth), _p(T_final), _p(last),
         _p(dL_drgb), _p(dL_ddepth), _p(dL_dT), _s(stream))


def gs_project_bwd(cfg, g: Gaussians, cams, ws, grads: dict, stream=None, overwrite=False):
    """Accumulates (+=) the gradients into ``grads`` or, with overwrite=True, stores them."""
    gs = g.struct()
    gr = GsGrads(*(_p(grads.get(k)) for k in ("means", "log_scales", "quats", "opacity_logits", "rgb", "pose")),
                 1 if overwrite else 0)
    call("gs_project_bwd", ctypes.byref(cfg), ctypes.byref(gs), _p(cams), _p(ws), ws.numel(), ctypes.byref(gr),
         _s(stream))


def gs_screen_grads(cfg, ws, d_mean2d=None, d_conic=None, d_depth=None, d_opacity=None, d_rgb=None, stream=None):
    call("gs_screen_grads", ctypes.byref(cfg), _p(ws), ws.numel(), _p(d_mean2d), _p(d_conic), _p(d_depth),
         _p(d_opacity), _p(d_rgb), _s(stream))


def gs_read_status(cfg, ws, stream=None):
    """Synchronises the stream; returns (status code, error word, total pairs, evals)."""
    err = ctypes.c_uint32()
    npairs = ctypes.c_int64()
    ev = ctypes.c_int64()
    code = _lib.load().gs_read_status(ctypes.byref(cfg), _p(ws), ws.numel(), ctypes.byref(err), ctypes.byref(npairs),
                                      ctypes.byref(ev), _s(stream))
    return code, err.value, npairs.value, ev.value


def gs_pose_adam_step(cams, pose_grad, state, lr_rho=1e-3, lr_phi=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                      zero_grad=True, stream=None):
    """One on-device Adam step of every view's pose from its se(3) gradient (cams updated in place)."""
    K = cams.shape[0]
    call("gs_pose_adam_step", _p(cams), _p(pose_grad), _p(state), ctypes.c_int32(K), ctypes.c_float(lr_rho),
         ctypes.c_float(lr_phi), ctypes.c_float(beta1), ctypes.c_float(beta2), ctypes.c_float(eps),
         ctypes.c_int32(1 if zero_grad else 0), _s(stream))


def gs_sort_pairs_tmp_size(n: int) -> int:
    b = ctypes.c_size_t()
    call("gs_sort_pairs_tmp_size", ctypes.c_int64(n), ctypes.byref(b))
    return b.value


def gs_sort_pairs(keys: torch.Tensor, vals: torch.Tensor, key_bits: int, tmp=None, err=None, stream=None):
    """In-place stable radix sort of int64 (bit pattern u64) keys with int32 (u32) values."""
    n = keys.numel()
    assert vals.numel() == n and keys.dtype == torch.int64 and vals.dtype == torch.int32
    if tmp is None:
        tmp = torch.empty(max(gs_sort_pairs_tmp_size(n), 256), dtype=torch.uint8, device=keys.device)
    call("gs_sort_pairs", _p(keys), _p(vals), ctypes.c_int64(n), ctypes.c_int32(key_bits), _p(tmp), tmp.numel(),
         _p(err), _s(stream))


def gs_sort_pairs_noalloc(keys: torch.Tensor, vals: torch.Tensor, key_bits: int, err=None, stream=None):
    """gs_sort_pairs without a temporary buffer (library-owned scratch, n <= SORT_NOALLOC_MAX_PAIRS)."""
    n = keys.numel()
    assert vals.numel() == n and keys.dtype == torch.int64 and vals.dtype == torch.int32
    call("gs_sort_pairs_noalloc", _p(keys), _p(vals), ctypes.c_int64(n), ctypes.c_int32(key_bits), _p(err),
         _s(stream))


# ----------------------------------------------------------------------------- the mapping loop

def gs_map_adam_state_size(N: int, color_width: int = 3) -> int:
    n = ctypes.c_int64()
    call("gs_map_adam_state_size", ctypes.c_int64(N), ctypes.c_int32(color_width), ctypes.byref(n))
    return n.value


def gs_map_adam_step(masters: "Gaussians", grads: dict, state: torch.Tensor, lr: dict, beta1=0.9, beta2=0.999,
                     eps=1e-15, storage: "Gaussians" = None, stream=None):
    """One Adam step of the FP32 master arrays from ``grads``; refreshes ``storage`` if given."""
    width = masters.rgb[0].numel() if masters.N else 3  # 3, or the SH coefficients' 3 (D+1)^2
    hp = GsAdam(lr["means"], lr["log_scales"], lr["quats"], lr["opacity_logits"], lr["rgb"], beta1, beta2, eps,
                width)
    gr = GsGrads(*(_p(grads.get(k)) for k in ("means", "log_scales", "quats", "opacity_logits", "rgb", "pose")), 0)
    st = storage.struct() if storage is not None else None
    call("gs_map_adam_step", ctypes.c_int64(masters.N), _p(masters.means), _p(masters.log_scales), _p(masters.quats),
         _p(masters.opacity_logits), _p(masters.rgb), ctypes.byref(gr), _p(state), ctypes.byref(hp),
         ctypes.byref(st) if st is not None else None, _s(stream))


def gs_keyframe_insert(cam: torch.Tensor, rgb, depth, T, out: "Gaussians", first: int, count: torch.Tensor,
                       stride=4, near=0.2, t_min=0.5, scale_factor=0.5, logit0=0.0, tmp=None, stream=None):
    """Appends one key-frame's new Gaussians to the FP32 arrays of ``out`` from index ``first``;
    ``count`` (a 1-element int32 device tensor) receives how many were written."""
    H, W = depth.shape[-2:]
    if tmp is None:
        b = ctypes.c_size_t()
        call("gs_keyframe_tmp_size", ctypes.c_int32(W), ctypes.c_int32(H), ctypes.c_int32(stride), ctypes.byref(b))
        tmp = torch.empty(b.value, dtype=torch.uint8, device=depth.device)
    call("gs_keyframe_insert", _p(cam), _p(rgb), _p(depth), _p(T), ctypes.c_int32(W), ctypes.c_int32(H),
         ctypes.c_int32(stride), ctypes.c_float(near), ctypes.c_float(t_min), ctypes.c_float(scale_factor),
         ctypes.c_float(logit0), _p(out.means), _p(out.log_scales), _p(out.quats), _p(out.opacity_logits),
         _p(out.rgb), ctypes.c_int64(first), ctypes.c_int64(out.N), _p(count), _p(tmp), tmp.numel(), _s(stream))


def _image_dims(x: torch.Tensor):
    if x.dim() == 3:
        x = x.unsqueeze(0)
    if x.dim() != 4 or x.dtype != torch.float32 or not x.is_contiguous():
        raise ValueError("images must be contiguous float32 [B, C, H, W] or [C, H, W]")
    return x.shape


def gs_metrics_tmp_size(images: int, channels: int, height: int, width: int) -> int:
    b = ctypes.c_size_t()
    call("gs_metrics_tmp_size", ctypes.c_int32(images), ctypes.c_int32(channels), ctypes.c_int32(height),
         ctypes.c_int32(width), ctypes.byref(b))
    return b.value


def gs_psnr(x: torch.Tensor, y: torch.Tensor, data_range=1.0, out=None, tmp=None, stream=None) -> torch.Tensor:
    """PSNR of each image of x against y ([B, C, H, W] or [C, H, W]); returns a device [B] tensor."""
    B, C, H, W = _image_dims(x)
    if tuple(y.shape[-3:]) != (C, H, W) or y.numel() != x.numel():
        raise ValueError("x and y must have the same shape")
    out = torch.empty(B, device=x.device) if out is None else out
    tmp = torch.empty(gs_metrics_tmp_size(B, C, H, W), dtype=torch.uint8, device=x.device) if tmp is None else tmp
    call("gs_psnr", _p(x), _p(y.contiguous()), ctypes.c_int32(B), ctypes.c_int32(C), ctypes.c_int32(H),
         ctypes.c_int32(W), ctypes.c_float(data_range), _p(out), _p(tmp), tmp.numel(), _s(stream))
    return out


def gs_ssim(x: torch.Tensor, y: torch.Tensor, data_range=1.0, out=None, ssim_map=None, tmp=None, stream=None):
    """Mean SSIM of each image of x against y; returns a device [B] tensor (and fills ssim_map,
    a [B, C, H, W] float32 tensor, when given)."""
    B, C, H, W = _image_dims(x)
    if tuple(y.shape[-3:]) != (C, H, W) or y.numel() != x.numel():
        raise ValueError("x and y must have the same shape")
    out = torch.empty(B, device=x.device) if out is None else out
    tmp = torch.empty(gs_metrics_tmp_size(B, C, H, W), dtype=torch.uint8, device=x.device) if tmp is None else tmp
    call("gs_ssim", _p(x), _p(y.contiguous()), ctypes.c_int32(B), ctypes.c_int32(C), ctypes.c_int32(H),
         ctypes.c_int32(W), ctypes.c_float(data_range), _p(out), _p(ssim_map), _p(tmp), tmp.numel(), _s(stream))
    return out


class MapOptimizer:
    """Adam over a map: FP32 master copies of the Gaussians (the render may read a reduced-storage
    copy, refreshed by every step), the optimiser state, the learning rates per group."""

    DEFAULT_LR = {"means": 1.6e-4, "log_scales": 5e-3, "quats": 1e-3, "opacity_logits": 5e-2, "rgb": 2.5e-3}

    def __init__(self, g: "Gaussians", lr: dict = None, beta1=0.9, beta2=0.999, eps=1e-15):
        f32 = lambda t: t.float().clone().contiguous()  # noqa: E731
        self.masters = Gaussians(f32(g.means), f32(g.log_scales), f32(g.quats), f32(g.opacity_logits), f32(g.rgb))
        all_f32 = all(t.dtype == torch.float32 for t in (g.means, g.log_scales, g.quats, g.opacity_logits, g.rgb))
        # an FP32 map is updated in place; a reduced-storage map is refreshed from the masters
        if all_f32:
            self.masters = g
            self.storage = None
        else:
            self.storage = g
        width = g.rgb[0].numel() if g.N else 3
        self.state = torch.zeros(gs_map_adam_state_size(g.N, width), device=g.means.device)
        self.lr = dict(self.DEFAULT_LR, **(lr or {}))
        self.beta1, self.beta2, self.eps = beta1, beta2, eps

    def step(self, grads: dict, stream=None):
        gs_map_adam_step(self.masters, grads, self.state, self.lr, self.beta1, self.beta2, self.eps, self.storage,
                         stream)


# ----------------------------------------------------------------------------- convenience

class CapacityOverflow(RuntimeError):
    pass


class Rasterizer:
    """Owns a workspace for (W, H, K views, N Gaussians) and chains the entry points.

    ``render`` runs gs_project -> gs_bin_sort -> gs_raster_fwd; ``backward`` runs
    gs_raster_bwd -> gs_project_bwd. Outputs and gradients are fresh torch tensors.
    """

    def __init__(self, width, height, num_views, num_gaussians, pair_capacity=None, device="cuda",
                 near_plane=0.2, lambda_depth=0.1, sh_degree=None):
        self.W, self.H, self.K, self.N = int(width), int(height), int(num_views), int(num_gaussians)
        self.device = torch.device(device)
        self.near_plane, self.lambda_depth = near_plane, lambda_depth
        self.sh_degree = sh_degree  # None: rgb [N,3] is the colour; 0..3: SH coefficients [N,(D+1)^2,3]
        if pair_capacity is None:
            pair_capacity = max(1 << 16, 8 * self.N * self.K)
        self._configure(pair_capacity)

    def _configure(self, cap):
        self.cap = int(min(cap, (1 << 30) - 1))
        old = getattr(self, "cfg", None)  # keep the tuned kernel variants across a capacity change
        tuned = (old.fwd_px_per_thread, old.bwd_px_per_thread, old.fwd_chunk, old.bwd_chunk) if old else (0, 0, 0, 0)
        self.cfg = make_config(self.W, self.H, self.K, self.N, self.cap, self.near_plane, self.lambda_depth, *tuned,
                               sh_degree=self.sh_degree, blocks_per_sm=old.raster_blocks_per_sm if old else 0)
        self.ws = workspace(self.cfg, self.device)
        self.layout = workspace_layout(self.cfg)

    def color_shape(self):
        """Shape of the Gaussians' rgb array (and of its gradient) for this rasterizer."""
        return (self.N, 3) if self.sh_degree is None else (self.N, (self.sh_degree + 1) ** 2, 3)

    def status(self, stream=None):
        return gs_read_status(self.cfg, self.ws, stream)

    def project_and_sort(self, g: Gaussians, cams: torch.Tensor, stream=None):
        gs_project(self.cfg, g, cams, self.ws, stream)
        gs_bin_sort(self.cfg, self.ws, stream)

    def plan(self, g: Gaussians, cams: torch.Tensor, headroom=1.25, stream=None) -> int:
        """Runs the projection and binning once and grows the pair capacity if needed."""
        self.project_and_sort(g, cams, stream)
        code, err, total, _ = self.status(stream)
        if err & _lib.DEVERR_PAIR_OVERFLOW:
            self._configure(int(total * headroom) + 1024)
            self.project_and_sort(g, cams, stream)
        return total

    def new_outputs(self):
        K, H, W, d = self.K, self.H, self.W, self.device
        return {"rgb": torch.empty((K, 3, H, W), device=d), "depth": torch.empty((K, H, W), device=d),
                "T": torch.empty((K, H, W), device=d), "last": torch.empty((K, H, W), dtype=torch.int32, device=d)}

    def render(self, g: Gaussians, cams: torch.Tensor, out=None, stream=None, stats=False):
        """stats=True also counts the evaluations and blended evaluations (``status()``)."""
        out = out or self.new_outputs()
        self.project_and_sort(g, cams, stream)
        fwd = gs_raster_fwd_stats if stats else gs_raster_fwd
        fwd(self.cfg, self.ws, out["rgb"], out["depth"], out["T"], out["last"], stream)
        return out

    def loss_l1(self, out, rgb_target, depth_target, stream=None):
        g_rgb = torch.empty_like(out["rgb"])
        g_depth = torch.empty_like(out["depth"])
        loss = torch.empty(1, device=self.device)
        gs_loss_l1(self.cfg, out["rgb"], out["depth"], rgb_target, depth_target, g_rgb, g_depth, loss, self.ws, stream)
        return loss, g_rgb, g_depth

    def backward(self, g: Gaussians, cams, out, dL_drgb, dL_ddepth, dL_dT=None, grads=None, stream=None):
        if grads is None:
            d = self.device
            grads = {"means": torch.zeros((self.N, 3), device=d), "log_scales": torch.zeros((self.N, 3), device=d),
                     "quats": torch.zeros((self.N, 4), device=d), "opacity_logits": torch.zeros(self.N, device=d),
                     "rgb": torch.zeros(self.color_shape(), device=d), "pose": torch.zeros((self.K, 6), device=d)}
        gs_raster_bwd(self.cfg, self.ws, out["rgb"], out["depth"], out["T"], out["last"], dL_drgb, dL_ddepth, dL_dT,
                      stream)
        gs_project_bwd(self.cfg, g, cams, self.ws, grads, stream)
        return grads

    def screen_grads(self, stream=None):
        d = self.device
        KN = self.K * self.N
        o = {"d_mean2d": torch.empty((KN, 2), device=d), "d_conic": torch.empty((KN, 3), device=d),
             "d_depth": torch.empty(KN, device=d), "d_opacity": torch.empty(self.N, device=d),
             "d_rgb": torch.empty((self.N, 3), device=d)}
        gs_screen_grads(self.cfg, self.ws, o["d_mean2d"], o["d_conic"], o["d_depth"], o["d_opacity"], o["d_rgb"],
                        stream)
        return o

    # --- workspace views (for inspection / tests) ---
    def ws_view(self, name, dtype, count):
        off = getattr(self.layout, name)
        nbytes = count * torch.empty((), dtype=dtype).element_size()
        return self.ws[off:off + nbytes].view(dtype)
