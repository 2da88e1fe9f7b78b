"""Autotuner for the compositing kernels.

The forward and backward compositing kernels come in variants that differ only in how
many pixels each thread owns (1, 2 or 4): every variant takes the same decisions (the
forward outputs are bit-identical, the gradients differ only in summation order), but
which is fastest depends on the image size, the number of views and how deep the tiles'
lists are. ``tune`` times each variant on the caller's own workspace (the
projection and binning of the real scene) with CUDA events and writes the fastest choice
into the rasterizer's config.
"""
from __future__ import annotations

import statistics

import torch

from . import api

VARIANTS = (1, 2, 4)


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
    """Chooses fwd_px_per_thread and bwd_px_per_thread for ``r`` (in place).

    Runs the projection and binning once, then times gs_raster_fwd and gs_raster_bwd for
    each variant with a fixed upstream gradient. Returns {"fwd": {px: ms}, "bwd": {px: ms},
    "choice": (fwd_px, bwd_px)}.
    """
    stream = stream if stream is not None else torch.cuda.current_stream()
    out = r.new_outputs()
    r.project_and_sort(g, cams, stream)
    api.gs_raster_fwd(r.cfg, r.ws, out["rgb"], out["depth"], out["T"], out["last"], stream)
    gen = torch.Generator(device=out["rgb"].device).manual_seed(0)
    g_rgb = torch.rand(out["rgb"].shape, generator=gen, device=out["rgb"].device) - 0.5
    g_depth = torch.rand(out["depth"].shape, generator=gen, device=out["depth"].device) - 0.5
    fwd, bwd = {}, {}
    saved = (r.cfg.fwd_px_per_thread, r.cfg.bwd_px_per_thread)
    for px in VARIANTS:
        r.cfg.fwd_px_per_thread = px
        fwd[px] = _time(lambda: api.gs_raster_fwd(r.cfg, r.ws, out["rgb"], out["depth"], out["T"], out["last"],
                                                  stream), reps, stream)
    for px in VARIANTS:
        r.cfg.bwd_px_per_thread = px
        bwd[px] = _time(lambda: api.gs_raster_bwd(r.cfg, r.ws, out["rgb"], out["depth"], out["T"], out["last"],
                                                  g_rgb, g_depth, None, stream), reps, stream)
    choice = (min(fwd, key=fwd.get), min(bwd, key=bwd.get))
    r.cfg.fwd_px_per_thread, r.cfg.bwd_px_per_thread = choice if all(choice) else saved
    return {"fwd": fwd, "bwd": bwd, "choice": choice}
