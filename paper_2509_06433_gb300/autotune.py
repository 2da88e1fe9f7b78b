"""Autotuner for the compositing kernels.

The forward and backward compositing kernels come in variants that differ in how many pixels
each thread owns (1, 2 or 4) and in how many splats a block stages in shared memory per step
(the chunk depth: 64, 128 or 256 for the forward, 32, 64 or 128 for the backward), and the
mapping step's forward + L1 loss + backward runs either as one launch (gs_raster_fwd_l1_bwd,
one pixels-per-thread value for both passes, the backward phase at a fixed chunk depth) or as
two; the chosen form then runs with a cap on its resident blocks per SM (none, 8, 6 or 4),
which trades occupancy for L1 cache and shared memory per block. When the one-launch form is
chosen, the forward-only paths (the viewer, plain renders) run at its pixels per thread and
chunk depth too. Every
variant takes the same decisions (the forward outputs are bit-identical, the gradients differ
only in summation order), but which is fastest depends on the image size, the number of views
and how deep the tiles' lists are. ``tune`` times each variant on the caller's own workspace
(the projection and binning of the real scene) with CUDA events and writes the fastest choice
into the rasterizer's config, and the one-or-two-launch choice into ``r.fused_compositing``.
(The tile size stays 16: the pairs are defined on 16x16 tiles.)
"""
from __future__ import annotations

import statistics

import torch

from . import api

PX = (1, 2, 4)
FWD_CHUNKS = (64, 128, 256)
BWD_CHUNKS = (32, 64, 128)
BLOCKS_PER_SM = (0, 8, 6, 4)  # cap on resident compositing blocks per SM (0: as many as fit)
FUSED_BWD_CHUNK = 64  # splats the backward phase of the one-launch form stages per chunk
VARIANTS = PX  # pixels-per-thread values (kept for callers that enumerate them)


def _time(fn, reps, stream):
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    fn()  # warm-up (first launch of a variant loads its module code)
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ev)


def tune(r: "api.Rasterizer", g: "api.Gaussians", cams: torch.Tensor, reps: int = 7, stream=None):
    """Chooses (pixels per thread, chunk depth) of gs_raster_fwd and gs_raster_bwd for ``r``.

    Runs the projection and binning once, then times every variant with a fixed upstream
    gradient; then the loss-fused forward followed by the backward (the chosen variants) against
    the one-launch form for each pixels-per-thread value (with that value's best forward chunk),
    against a zero target. Returns {"fwd": {(px, chunk): ms}, "bwd": {(px, chunk): ms},
    "choice": (fwd_px, bwd_px), "chunks": (fwd_chunk, bwd_chunk in use), "two_launch_ms": ms,
    "fused_ms": {(px, chunk): ms}, "fused": bool, "blocks_per_sm_ms": {cap: ms}, "blocks_per_sm": cap}.
    """
    stream = stream if stream is not None else torch.cuda.current_stream()
    out = r.new_outputs()
    r.project_and_sort(g, cams, stream)
    api.gs_raster_fwd(r.cfg, r.ws, out["rgb"], out["depth"], out["T"], out["last"], stream)
    gen = torch.Generator(device=out["rgb"].device).manual_seed(0)
    g_rgb = torch.rand(out["rgb"].shape, generator=gen, device=out["rgb"].device) - 0.5
    g_depth = torch.rand(out["depth"].shape, generator=gen, device=out["depth"].device) - 0.5
    fwd, bwd = {}, {}
    c = r.cfg
    saved = (c.fwd_px_per_thread, c.bwd_px_per_thread, c.fwd_chunk, c.bwd_chunk)
    c.raster_blocks_per_sm = 0  # the variants are compared without a cap
    for px in PX:
        for ch in FWD_CHUNKS:
            c.fwd_px_per_thread, c.fwd_chunk = px, ch
            fwd[(px, ch)] = _time(lambda: api.gs_raster_fwd(c, r.ws, out["rgb"], out["depth"], out["T"], out["last"],
                                                            stream), reps, stream)
    for px in PX:
        for ch in BWD_CHUNKS:
            c.bwd_px_per_thread, c.bwd_chunk = px, ch
            bwd[(px, ch)] = _time(lambda: api.gs_raster_bwd(c, r.ws, out["rgb"], out["depth"], out["T"], out["last"],
                                                            g_rgb, g_depth, None, stream), reps, stream)
    fbest, bbest = min(fwd, key=fwd.get), min(bwd, key=bwd.get)
    c.fwd_px_per_thread, c.fwd_chunk = fbest
    c.bwd_px_per_thread, c.bwd_chunk = bbest
    if not all(fbest + bbest):
        c.fwd_px_per_thread, c.bwd_px_per_thread, c.fwd_chunk, c.bwd_chunk = saved
    # the mapping step's compositing: two launches with the choices above, or one
    rgb_t, depth_t = torch.zeros_like(out["rgb"]), torch.zeros_like(out["depth"])
    lg_rgb, lg_depth = torch.empty_like(out["rgb"]), torch.empty_like(out["depth"])
    loss = torch.empty(1, device=out["rgb"].device)
    imgs = (out["rgb"], out["depth"], out["T"], out["last"])

    def two_launches():
        api.gs_raster_fwd_l1(c, r.ws, *imgs, rgb_t, depth_t, lg_rgb, lg_depth, loss, stream)
        api.gs_raster_bwd(c, r.ws, *imgs, lg_rgb, lg_depth, None, stream)

    two = _time(two_launches, reps, stream)
    chosen = (c.fwd_px_per_thread, c.bwd_px_per_thread, c.fwd_chunk)
    fused = {}
    for px in PX:
        ch = min((k for k in fwd if k[0] == px), key=fwd.get)[1]
        c.fwd_px_per_thread = c.bwd_px_per_thread = px
        c.fwd_chunk = ch
        fused[(px, ch)] = _time(lambda: api.gs_raster_fwd_l1_bwd(c, r.ws, *imgs, rgb_t, depth_t, lg_rgb, lg_depth,
                                                                 loss, stream), reps, stream)
    c.fwd_px_per_thread, c.bwd_px_per_thread, c.fwd_chunk = chosen
    fb = min(fused, key=fused.get)
    r.fused_compositing = bool(fused[fb] < two)
    if r.fused_compositing:
        c.fwd_px_per_thread = c.bwd_px_per_thread = fb[0]
        c.fwd_chunk = fb[1]
    # blocks per SM of the chosen form: fewer resident blocks give each more L1 / shared memory
    step = (lambda: api.gs_raster_fwd_l1_bwd(c, r.ws, *imgs, rgb_t, depth_t, lg_rgb, lg_depth, loss, stream)) \
        if r.fused_compositing else two_launches
    bps = {}
    for b in BLOCKS_PER_SM:
        c.raster_blocks_per_sm = b
        bps[b] = _time(step, reps, stream)
    c.raster_blocks_per_sm = min(bps, key=bps.get)
    return {"fwd": fwd, "bwd": bwd, "choice": (c.fwd_px_per_thread, c.bwd_px_per_thread),
            # the one-launch form's backward phase stages FUSED_BWD_CHUNK splats whatever bwd_chunk says
            "chunks": (c.fwd_chunk, FUSED_BWD_CHUNK if r.fused_compositing else c.bwd_chunk),
            "two_launch_ms": two, "fused_ms": fused, "fused": r.fused_compositing,
            "blocks_per_sm_ms": bps, "blocks_per_sm": c.raster_blocks_per_sm}
