"""Render-based camera tracking and CUDA-graph-captured iterations.

A tracking iteration renders the fixed Gaussian map at the current pose estimate,
compares it with the observed frame (L1 on RGB + lambda L1 on depth), back-propagates
to the se(3) pose only, and takes one Adam step on the pose (T <- Exp(xi) T), all on
the device. ``Tracker`` captures one iteration in a CUDA graph and replays it, so an
iteration costs one graph launch and no host round trip.

``MappingStep`` does the same for a mapping iteration (fixed poses, gradients for every
Gaussian parameter), so the K-view forward + backward of a mapping window replays as one
graph.
"""
from __future__ import annotations

import torch

from . import api


def fuses_backward(r) -> bool:
    """Whether the rasterizer's forward and backward compositing run as one launch
    (gs_raster_fwd_l1_bwd): only when both use the same pixels per thread (then the results are
    those of the two calls bit for bit), and not when the autotuner found two launches faster
    (``r.fused_compositing``)."""
    px = lambda v: v if v in (1, 2, 4) else 2  # noqa: E731  (0 = the library default, 2)
    c = r.cfg
    return px(c.fwd_px_per_thread) == px(c.bwd_px_per_thread) and getattr(r, "fused_compositing", True)


def fwd_l1_bwd(r, out, rgb_t, depth_t, g_rgb, g_depth, loss, stream=None):
    """Forward with the fused L1 loss, then the backward compositing: one launch
    (gs_raster_fwd_l1_bwd) when fuses_backward(r), else gs_raster_fwd_l1 + gs_raster_bwd."""
    c = r.cfg
    args = (c, r.ws, out["rgb"], out["depth"], out["T"], out["last"])
    if fuses_backward(r):
        api.gs_raster_fwd_l1_bwd(*args, rgb_t, depth_t, g_rgb, g_depth, loss, stream)
    else:
        api.gs_raster_fwd_l1(*args, rgb_t, depth_t, g_rgb, g_depth, loss, stream)
        api.gs_raster_bwd(*args, g_rgb, g_depth, None, stream)


class _Captured:
    def __init__(self, graph: bool):
        self.use_graph = graph
        self.graph = None

    def _capture(self, body, warmup=2):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):  # first launches set kernel attributes outside the capture
                body()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        if self.use_graph:
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                body()
        self._body = body

    def replay(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self._body()


class Tracker(_Captured):
    """Pose tracking of K views against observed frames with a fixed map.

    cams: [K,16] float32 CUDA tensor (updated in place by every iteration); rgb_obs
    [K,3,H,W] and depth_obs [K,H,W]: the observed frames.
    """

    def __init__(self, g: api.Gaussians, cams: torch.Tensor, width: int, height: int, rgb_obs: torch.Tensor,
                 depth_obs: torch.Tensor, lr_rho=2e-3, lr_phi=2e-3, lambda_depth=0.1, pair_headroom=1.5,
                 graph=True, autotune=False):
        super().__init__(graph)
        self.g, self.cams = g, cams
        K = cams.shape[0]
        self.r = api.Rasterizer(width, height, K, g.N, device=cams.device, lambda_depth=lambda_depth)
        total = self.r.plan(g, cams)
        if total * pair_headroom > self.r.cap:
            self.r._configure(int(total * pair_headroom) + 4096)
        if autotune:
            from . import autotune as at
            at.tune(self.r, g, cams)
        self.rgb_obs, self.depth_obs = rgb_obs, depth_obs
        self.out = self.r.new_outputs()
        d = cams.device
        self.g_rgb = torch.empty_like(self.out["rgb"])
        self.g_depth = torch.empty_like(self.out["depth"])
        self.loss = torch.zeros(1, device=d)
        self.pose_grad = torch.zeros((K, 6), device=d)
        self.state = torch.zeros((K, 16), device=d)
        self.lr = (lr_rho, lr_phi)
        start = cams.clone()
        self._capture(self._iteration)
        cams.copy_(start)  # the warm-up iterations moved the pose: start from the given one
        self.reset_optimizer()

    def _iteration(self):
        r, o = self.r, self.out
        api.gs_project(r.cfg, self.g, self.cams, r.ws)
        api.gs_bin_sort(r.cfg, r.ws)
        fwd_l1_bwd(r, o, self.rgb_obs, self.depth_obs, self.g_rgb, self.g_depth, self.loss)
        api.gs_project_bwd(r.cfg, self.g, self.cams, r.ws, {"pose": self.pose_grad}, overwrite=True)
        api.gs_pose_adam_step(self.cams, self.pose_grad, self.state, self.lr[0], self.lr[1], zero_grad=False)

    def reset_optimizer(self):
        self.state.zero_()
        self.pose_grad.zero_()

    def run(self, iters: int):
        for _ in range(iters):
            self.replay()
        return self.cams

    def status(self):
        return self.r.status()


class MappingStep(_Captured):
    """One mapping iteration (fixed poses): render with the L1 loss against the key-frames fused
    into the forward pass, backward to every Gaussian parameter and the poses (the gradients
    are stored, not accumulated, so nothing is zeroed), and, with an ``optimizer``, its Adam
    step of the map; the whole iteration is one CUDA graph."""

    def __init__(self, r: api.Rasterizer, g: api.Gaussians, cams: torch.Tensor, rgb_t: torch.Tensor,
                 depth_t: torch.Tensor, graph=True, optimizer: "api.MapOptimizer" = None):
        super().__init__(graph)
        self.r, self.g, self.cams, self.rgb_t, self.depth_t = r, g, cams, rgb_t, depth_t
        self.optimizer = optimizer
        d = cams.device
        N, K = g.N, cams.shape[0]
        self.out = r.new_outputs()
        self.g_rgb = torch.empty_like(self.out["rgb"])
        self.g_depth = torch.empty_like(self.out["depth"])
        self.grads, self.loss = self._alloc_grads(r, N, K, d)
        saved = self._snapshot()
        self._capture(self._iteration)
        self._restore(saved)  # the warm-up iterations stepped the optimiser: start from the given map

    @staticmethod
    def _alloc_grads(r, N, K, d):
        grads = {"means": torch.zeros((N, 3), device=d), "log_scales": torch.zeros((N, 3), device=d),
                 "quats": torch.zeros((N, 4), device=d), "opacity_logits": torch.zeros(N, device=d),
                 "rgb": torch.zeros(r.color_shape(), device=d), "pose": torch.zeros((K, 6), device=d)}
        return grads, torch.zeros(1, device=d)

    def _tensors(self):
        if self.optimizer is None:
            return []
        o = self.optimizer
        ts = [o.state] + [getattr(o.masters, k) for k in ("means", "log_scales", "quats", "opacity_logits", "rgb")]
        if o.storage is not None:
            ts += [getattr(o.storage, k) for k in ("means", "log_scales", "quats", "opacity_logits", "rgb")]
        return ts

    def _snapshot(self):
        return [t.clone() for t in self._tensors()]

    def _restore(self, saved):
        for t, c in zip(self._tensors(), saved):
            t.copy_(c)

    def _iteration(self):
        r, o = self.r, self.out
        api.gs_project(r.cfg, self.g, self.cams, r.ws)
        api.gs_bin_sort(r.cfg, r.ws)
        fwd_l1_bwd(r, o, self.rgb_t, self.depth_t, self.g_rgb, self.g_depth, self.loss)
        api.gs_project_bwd(r.cfg, self.g, self.cams, r.ws, self.grads, overwrite=True)
        if self.optimizer is not None:
            self.optimizer.step(self.grads)


class HostMappingStep(MappingStep):
    """A mapping iteration fed from host memory, for callers whose map and key-frames live on
    the host: every replay copies the Gaussians, the cameras and the key-frame targets from
    pinned host buffers to the device, runs the iteration (render with the fused L1 loss,
    backward to every parameter and the poses) and copies the gradients and the loss back to
    pinned host buffers; copies and kernels are one CUDA graph.

    The Gaussians (in their storage precision) and cameras travel as one packed buffer and the
    gradients with the loss as one, so a replay makes three host-to-device copies (the packed inputs first; then
    the targets on a side stream, overlapping the projection and binning) and one
    device-to-host copy.

    Fill the tensors of ``host_in`` (views of the pinned buffers: the five Gaussian arrays,
    ``cams``, ``rgb_t``, ``depth_t``) before ``replay()``; ``host_out`` (the gradients and
    ``loss``) is valid once the stream has synchronised."""

    _IN = ("means", "log_scales", "quats", "opacity_logits", "rgb", "cams")

    def __init__(self, r: api.Rasterizer, host_gaussians: api.Gaussians, host_cams: torch.Tensor,
                 host_rgb_t: torch.Tensor, host_depth_t: torch.Tensor, graph=True):
        d = torch.device("cuda", torch.cuda.current_device()) if r.device.index is None else r.device
        src = {k: getattr(host_gaussians, k) for k in self._IN[:5]}
        src["cams"] = host_cams.float()
        # one byte buffer holds every input in its own dtype (the Gaussians in their storage
        # precision), each array starting on a 256-byte boundary
        offs, off = {}, 0
        for k in self._IN:
            offs[k] = off
            off += (src[k].numel() * src[k].element_size() + 255) // 256 * 256
        self._h_pack = torch.empty(off, dtype=torch.uint8, pin_memory=True)
        self._d_pack = torch.empty(off, dtype=torch.uint8, device=d)
        self.host_in, self.dev_in = {}, {}
        for k in self._IN:
            v = src[k]
            n = v.numel() * v.element_size()
            self.host_in[k] = self._h_pack[offs[k]:offs[k] + n].view(v.dtype).view(v.shape)
            self.dev_in[k] = self._d_pack[offs[k]:offs[k] + n].view(v.dtype).view(v.shape)
            self.host_in[k].copy_(v)
        for k, v in (("rgb_t", host_rgb_t), ("depth_t", host_depth_t)):
            self.host_in[k] = v.contiguous().float().pin_memory()
            self.dev_in[k] = torch.empty_like(self.host_in[k], device=d)
        self._d_pack.copy_(self._h_pack)
        for k in ("rgb_t", "depth_t"):
            self.dev_in[k].copy_(self.host_in[k])
        self._side = torch.cuda.Stream(device=d)
        g = api.Gaussians(*(self.dev_in[k] for k in self._IN[:5]))
        super().__init__(r, g, self.dev_in["cams"], self.dev_in["rgb_t"], self.dev_in["depth_t"], graph=graph)

    def _alloc_grads(self, r, N, K, d):
        # gradients and loss as views of one device buffer, mirrored by one pinned host buffer
        shapes = {"means": (N, 3), "log_scales": (N, 3), "quats": (N, 4), "opacity_logits": (N,),
                  "rgb": tuple(r.color_shape()), "pose": (K, 6), "loss": (1,)}
        total = sum(int(torch.Size(v).numel()) for v in shapes.values())
        self._d_out = torch.zeros(total, device=d)
        self._h_out = torch.zeros(total, pin_memory=True)
        views, self.host_out, off = {}, {}, 0
        for k, shp in shapes.items():
            n = int(torch.Size(shp).numel())
            views[k] = self._d_out[off:off + n].view(shp)
            self.host_out[k] = self._h_out[off:off + n].view(shp)
            off += n
        loss = views.pop("loss")
        return views, loss

    def _iteration(self):
        r, o = self.r, self.out
        main = torch.cuda.current_stream()
        # the Gaussians and cameras go first, alone on the link; the key-frame targets, needed
        # only by the forward, follow on a side stream while the projection and binning run
        self._d_pack.copy_(self._h_pack, non_blocking=True)
        self._side.wait_stream(main)
        with torch.cuda.stream(self._side):
            for k in ("rgb_t", "depth_t"):
                self.dev_in[k].copy_(self.host_in[k], non_blocking=True)
        api.gs_project(r.cfg, self.g, self.cams, r.ws)
        api.gs_bin_sort(r.cfg, r.ws)
        main.wait_stream(self._side)
        fwd_l1_bwd(r, o, self.rgb_t, self.depth_t, self.g_rgb, self.g_depth, self.loss)
        api.gs_project_bwd(r.cfg, self.g, self.cams, r.ws, self.grads, overwrite=True)
        self._h_out.copy_(self._d_out, non_blocking=True)

    def transfer_bytes(self):
        """(host-to-device, device-to-host) bytes per replay."""
        h2d = self._h_pack.numel() + 4 * (self.host_in["rgb_t"].numel() + self.host_in["depth_t"].numel())
        return h2d, 4 * self._h_out.numel()
