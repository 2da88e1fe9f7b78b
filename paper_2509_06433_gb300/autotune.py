"""Autotuner for the compositing kernels.

The forward and backward compositing kernels come in variants that differ in how many pixels
each thread owns (1, 2 or 4) and in how many splats a block stages in shared memory per step
(the chunk depth: 64, 128 or 256 for the forward, 32, 64 or 128 for the backward). Every
variant takes the same decisions (the forward outputs are bit-identical, the gradients differ
only in summation order), but which is fastest depends on the image size, the number of views
and how deep the tiles' lists are. ``tune`` times each variant on the caller's own workspace
(the projection and binning of the real scene) with CUDA events and writes the fastest choice
into the rasterizer's config. (The tile size stays 16: the pairs are defined on 16x16 tiles.)
"""
from __future__ import annotations

import statistics

import torch

from . import api

PX = (1, 2, 4)
FWD_CHUNKS = (64, 128, 256)
BWD_CHUNKS = (32, 64, 128)
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
    gradient. Returns {"fwd": {(px, chunk): ms}, "bwd": {(px, chunk): ms},
    "choice": (fwd_px, bwd_px), "chunks": (fwd_chunk, bwd_chunk)}.
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
    return {"fwd": fwd, "bwd": bwd, "choice": (fbest[0], bbest[0]), "chunks": (fbest[1], bbest[1])}
