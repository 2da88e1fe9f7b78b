"""Online mapping from a stream of RGB-D key-frames (the mapping side of Fig. 3).

Each incoming key-frame is first rendered from the current map; its pixels that the map
does not yet cover (transmittance above ``t_min``) become new Gaussians
(gs_keyframe_insert). Mapping iterations then optimise the whole map against a sliding
window of the latest ``window`` key-frames: one CUDA graph per iteration holding the
K-view render with the fused L1 loss, the backward pass and the Adam step
(tracking.MappingStep with an api.MapOptimizer).

The map lives in FP32 arrays of a fixed ``capacity``; slots not filled yet hold Gaussians
with opacity logit -30 (opacity ~1e-13, below 1/255 everywhere: they touch no tile and get
zero gradients, so Adam leaves them unchanged). The mapping graph is built once and
replayed; a new key-frame only rewrites the window's camera and target buffers in place.
"""
from __future__ import annotations

import torch

from . import api
from .tracking import MappingStep

EMPTY_LOGIT = -30.0


class OnlineMapper:
    def __init__(self, width: int, height: int, capacity: int, window: int = 4, lr: dict = None, stride: int = 4,
                 t_min: float = 0.5, scale_factor: float = 0.5, logit0: float = 0.0, lambda_depth: float = 0.1,
                 pairs_per_gaussian: int = 12, graph: bool = True, device="cuda"):
        self.W, self.H, self.capacity, self.window = int(width), int(height), int(capacity), int(window)
        self.stride, self.t_min, self.scale_factor, self.logit0 = stride, t_min, scale_factor, logit0
        self.graph = graph
        d = self.device = torch.device(device)
        C = self.capacity
        quats = torch.zeros((C, 4), device=d)
        quats[:, 0] = 1.0
        self.g = api.Gaussians(torch.zeros((C, 3), device=d), torch.full((C, 3), -5.0, device=d), quats,
                               torch.full((C,), EMPTY_LOGIT, device=d), torch.zeros((C, 3), device=d))
        self.count = 0
        self.frames = 0
        self.opt = api.MapOptimizer(self.g, lr)
        self.cams = torch.zeros((window, 16), device=d)
        self.rgb_t = torch.zeros((window, 3, height, width), device=d)
        self.depth_t = torch.zeros((window, height, width), device=d)
        cap = pairs_per_gaussian * C * window
        self.r = api.Rasterizer(width, height, window, C, pair_capacity=cap, device=d, lambda_depth=lambda_depth)
        self.view = api.Rasterizer(width, height, 1, C, pair_capacity=pairs_per_gaussian * C, device=d)
        self._n_new = torch.zeros(1, dtype=torch.int32, device=d)
        # the mapping graph is captured once here (on the empty map and zero targets) and
        # replayed; it is rebuilt only when the pair capacity has to grow
        self.step = MappingStep(self.r, self.g, self.cams, self.rgb_t, self.depth_t, graph=graph, optimizer=self.opt)
        self._warm_up()

    def _warm_up(self):
        """First launches of the single-view render and of the insertion kernels (module loading,
        kernel attributes) happen here rather than inside the first key-frame's time: a render
        of the empty map and an insertion from a frame without valid depth (adds nothing)."""
        cam = torch.zeros(16, device=self.device)
        cam[0] = cam[1] = float(max(self.W, self.H))
        cam[2], cam[3] = self.W / 2.0, self.H / 2.0
        cam[4] = cam[8] = cam[12] = 1.0
        T = self.render(cam)["T"][0]
        api.gs_keyframe_insert(cam.reshape(1, 16), torch.zeros((3, self.H, self.W), device=self.device),
                               torch.zeros((self.H, self.W), device=self.device), T, self.g, self.count,
                               self._n_new, stride=self.stride, t_min=self.t_min)
        api.gs_psnr(self.rgb_t[:1], self.rgb_t[:1])
        api.gs_ssim(self.rgb_t[:1], self.rgb_t[:1])
        torch.cuda.synchronize()

    # ------------------------------------------------------------------ key-frames
    def add_keyframe(self, rgb: torch.Tensor, depth: torch.Tensor, cam: torch.Tensor) -> int:
        """rgb [3,H,W], depth [H,W] (metric depth, <= near where invalid), cam [16]: inserts the
        frame's uncovered pixels as Gaussians and makes the frame the newest of the window.
        Returns the number of Gaussians added (this call reads it back: one host sync)."""
        cam = cam.reshape(1, 16).contiguous()
        T = self.render(cam)["T"][0]
        api.gs_keyframe_insert(cam, rgb.contiguous(), depth.contiguous(), T, self.g, self.count, self._n_new,
                               stride=self.stride, t_min=self.t_min, scale_factor=self.scale_factor,
                               logit0=self.logit0)
        added = int(self._n_new.item())
        self.count += added
        # window: slot i holds the i-th newest frame; before the window is full, the newest
        # frame fills the remaining slots as well
        self.cams.copy_(torch.roll(self.cams, 1, 0))
        self.rgb_t.copy_(torch.roll(self.rgb_t, 1, 0))
        self.depth_t.copy_(torch.roll(self.depth_t, 1, 0))
        self.frames += 1
        fill = self.window if self.frames == 1 else 1
        self.cams[:fill] = cam
        self.rgb_t[:fill] = rgb
        self.depth_t[:fill] = depth  # the loss compares it with the rendered depth sum(z w)
        self._ensure_capacity()
        return added

    def _ensure_capacity(self):
        """Grows the window rasterizer's pair capacity if the current map needs it (and then
        rebuilds the mapping graph, which holds the workspace's address)."""
        cap0 = self.r.cap
        self.r.plan(self.g, self.cams, headroom=1.5)
        if self.r.cap != cap0:
            self.step = MappingStep(self.r, self.g, self.cams, self.rgb_t, self.depth_t, graph=self.graph,
                                    optimizer=self.opt)

    # ------------------------------------------------------------------ mapping
    def iterate(self, n: int):
        for _ in range(n):
            self.step.replay()

    def overflowed(self) -> bool:
        _, err, _, _ = self.r.status()
        return bool(err & 0x1)

    def render(self, cam: torch.Tensor, out=None):
        cam = cam.reshape(1, 16).contiguous()
        self.view.plan(self.g, cam, headroom=1.5)
        return self.view.render(self.g, cam, out)


def evaluate(mapper: OnlineMapper, rgb: torch.Tensor, cam: torch.Tensor):
    """PSNR and SSIM (GPU reductions) of the map rendered at cam against the frame rgb [3,H,W]."""
    out = mapper.render(cam)
    x, y = out["rgb"], rgb.reshape(1, *rgb.shape[-3:]).contiguous()
    return float(api.gs_psnr(x, y)[0]), float(api.gs_ssim(x, y)[0])


def map_sequence(mapper: OnlineMapper, frames, iters_per_frame=200, eval_every=10, thresholds=(20.0, 21.0)):
    """Map a key-frame sequence as it arrives and record how fast each frame's view converges.

    frames: (rgb [3,H,W], depth [H,W], cam [16]) device tensors in arrival order. For each frame:
    insert it, then run ``iters_per_frame`` mapping iterations in blocks of ``eval_every``. The
    mapping time (insertion included, the evaluations excluded) is taken with CUDA events; the
    frame's PSNR / SSIM is evaluated before the first block and after every block. Returns one
    record per frame: Gaussians added, the (seconds, iterations, PSNR, SSIM) curve, and the
    seconds at which the PSNR first reached each threshold (None if it did not)."""
    records = []
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for j, (rgb, depth, cam) in enumerate(frames):
        a.record()
        added = mapper.add_keyframe(rgb, depth, cam)
        b.record()
        b.synchronize()
        t = a.elapsed_time(b) / 1e3
        p, s = evaluate(mapper, rgb, cam)
        curve = [(t, 0, p, s)]
        for blk in range(iters_per_frame // eval_every):
            a.record()
            mapper.iterate(eval_every)
            b.record()
            b.synchronize()
            t += a.elapsed_time(b) / 1e3
            p, s = evaluate(mapper, rgb, cam)
            curve.append((t, (blk + 1) * eval_every, p, s))
        reach = {thr: next((c[0] for c in curve if c[2] >= thr), None) for thr in thresholds}
        records.append({"frame": j, "added": added, "gaussians": mapper.count, "curve": curve, "t_reach": reach})
    return records
