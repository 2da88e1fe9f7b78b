"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and
read its outputs back as numpy; compare against the oracle with the tolerances of
the method (keys, order, ranges and rectangles bit-exact; images max-abs 1e-4;
gradients relative L2 1e-3)."""
from __future__ import annotations

import numpy as np

IMG_ATOL = 1e-4       # max-abs tolerance of RGB, depth and T against the FP64 oracle
GRAD_RTOL = 1e-3      # relative L2 tolerance of every gradient tensor
MAX_EXCLUDED = 1e-3   # fraction of pixels with >= 2 near-threshold decisions allowed out of the check


def torch_mods():
    import torch
    from paper_2509_06433_gb300 import api
    return torch, api


def cams_tensor(cams):
    torch, _ = torch_mods()
    return torch.as_tensor(np.ascontiguousarray(np.asarray(cams, np.float32).reshape(-1, 16))).cuda()


def gpu_render(params, cams, W, H, cap=None, dtype=None, means_dtype=None):
    """Projection + binning + forward raster on the GPU. Returns (rasterizer, gaussians, cams, outputs)."""
    torch, api = torch_mods()
    dtype = dtype or torch.float32
    means_dtype = means_dtype or torch.float32
    g = api.Gaussians.from_numpy(params, dtype=dtype, means_dtype=means_dtype)
    ct = cams_tensor(cams)
    r = api.Rasterizer(W, H, ct.shape[0], g.N, pair_capacity=cap)
    r.plan(g, ct)
    out = r.render(g, ct, stats=True)
    torch.cuda.synchronize()
    return r, g, ct, out


def read_discrete(r):
    """Projection records, sorted pairs and ranges from the workspace."""
    torch, _ = torch_mods()
    code, err, total, evals = r.status()
    KN = r.K * r.N
    lay = r.layout
    # items that emit pairs (live); the projection records exist for those only
    mask = r.ws_view("live_mask", torch.int32, (KN + 31) // 32).cpu().numpy().view(np.uint32)
    live = ((mask[np.arange(KN) >> 5] >> (np.arange(KN) & 31).astype(np.uint32)) & 1).astype(bool)
    tiles = r.ws_view("proj_tiles", torch.int32, KN * 4).reshape(KN, 4).cpu().numpy()
    tiles[~live] = 0
    # a live item's first pair index, stored at its rank among the live items
    n_live = int(live.sum())
    tiles[live, 0] = r.ws_view("live_off", torch.int32, max(n_live, 1)).cpu().numpy()[:n_live]
    rx = tiles[:, 1].view(np.uint32)
    ry = tiles[:, 2].view(np.uint32)
    rect = np.stack([rx & 0xFFFF, rx >> 16, ry & 0xFFFF, ry >> 16], axis=1).astype(np.int32)
    P = min(total, r.cap)
    # the sorted pairs carry (tile << 32) | Gaussian id and, as value, the pair's emission
    # index; rebuild the (tile << 32) | depth-bits keys and Gaussian-id values of the method
    raw_keys = r.ws_view("keys_sorted", torch.int64, P).cpu().numpy().view(np.uint64)
    raw_vals = r.ws_view("vals_sorted", torch.int32, P).cpu().numpy().view(np.uint32)
    depth_bits = r.ws_view("proj_depth_key", torch.int32, KN).cpu().numpy().view(np.uint32)
    tile = raw_keys >> np.uint64(32)
    gid = (raw_keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    item = (tile // np.uint64(lay.tiles_x * lay.tiles_y)).astype(np.int64) * r.N + gid
    keys = (tile << np.uint64(32)) | depth_bits[item].astype(np.uint64) if P else raw_keys
    d = {
        "status": code, "err": err, "total_pairs": total, "evals": evals,
        "live": live,
        "offset": tiles[:, 0].copy(), "count": tiles[:, 3].view(np.uint32).copy(), "rect": rect,
        "depth_bits": depth_bits,
        "radius": np.where(live, r.ws_view("proj_radius", torch.int32, KN).cpu().numpy(), 0),
        "uv": r.ws_view("proj_uv", torch.float32, KN * 4).reshape(KN, 4).cpu().numpy(),
        "conic": r.ws_view("proj_conic", torch.float32, KN * 4).reshape(KN, 4).cpu().numpy(),
        "keys": keys, "vals": gid.astype(np.uint32), "slots": raw_vals, "item": item,
        "ranges": r.ws_view("ranges", torch.int32, r.K * lay.tiles_x * lay.tiles_y * 2).reshape(-1, 2).cpu()
        .numpy().view(np.uint32),
    }
    return d


def to_np(out):
    return {k: v.detach().cpu().numpy() for k, v in out.items()}


def check_images(gpu, orc, atol=IMG_ATOL, max_excluded=MAX_EXCLUDED):
    """Element-wise image parity. A pixel whose oracle list holds exactly one decision in the
    guard band of a threshold passes if it matches either the primary or the alternative
    oracle result; pixels with two or more such decisions are excluded and counted."""
    near = orc["near"]
    excluded = near >= 2
    assert excluded.mean() <= max_excluded, f"excluded fraction {excluded.mean():.2e}"
    report = {}
    for key, okey in (("rgb", "rgb"), ("depth", "depth"), ("T", "T")):
        a = gpu[key].astype(np.float64)
        p = np.abs(a - orc[okey])
        q = np.abs(a - orc["alt_" + okey])
        if key == "rgb":
            nb = np.broadcast_to(near[:, None], p.shape)
            ex = np.broadcast_to(excluded[:, None], p.shape)
        else:
            nb, ex = near, excluded
        ok = (p <= atol) | ((nb == 1) & (q <= atol)) | ex
        bad = np.argwhere(~ok)
        assert bad.size == 0, (f"{key}: {len(bad)} elements off; first {bad[:5].tolist()} "
                               f"gpu {a[tuple(bad[0])]:.7g} oracle {orc[okey][tuple(bad[0])]:.7g}")
        report[key] = float(np.where(near == 0 if key != "rgb" else (near == 0)[:, None], p, 0).max())
    last_ok = (gpu["last"] == orc["last"]) | ((near == 1) & (gpu["last"] == orc["alt_last"])) | excluded
    assert last_ok.all(), f"last differs at {np.argwhere(~last_ok)[:5].tolist()}"
    report["near_pixels"] = int((near > 0).sum())
    report["excluded"] = int(excluded.sum())
    return report


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a))
