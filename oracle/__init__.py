"""FP64 CPU oracle of the differentiable Gaussian rasterizer (ctypes wrapper).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The CUDA library and its Python binding never do, and this package
never imports them.

Every function takes numpy arrays. Continuous inputs are converted exactly to
float64 (a float32, bfloat16 or float16 stored value is exactly representable
in float64), so the oracle sees the same numbers as the GPU path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

#: thresholds of the method reading (kept here only to size guard bands in reports)
NEAR = 0.2
TILE = 16

#: default guard half-widths (relative) around the alpha >= 1/255 test, the
#: T(1-alpha) < 1e-4 stop and the power > 0 test: a decision whose value lies within
#: this band of its threshold is flagged, and the pixel is also rendered with it inverted.
GUARD_ALPHA = 2e-5
GUARD_T = 2e-4
GUARD_POWER = 1e-5


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (g++, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double
_F = ctypes.c_float


def _declare(L):
    L.orc_expdet_f32.argtypes = [_P, _P, _I64]
    L.orc_expdet_f32.restype = None
    L.orc_logdet_f32.argtypes = [_P, _P, _I64]
    L.orc_logdet_f32.restype = None
    L.orc_project_mirror.argtypes = [_I64, _P, _P, _P, _P, _I, _P, _I, _I, _I, _F, _P, _P, _P, _P, _P, _P]
    L.orc_project_mirror.restype = None
    L.orc_project64.argtypes = [_I64, _P, _P, _P, _P, _P, _I, _P, _I, _I, _P]
    L.orc_project64.restype = None
    L.orc_render_occluded.argtypes = [_I64, _P, _P, _P, _P, _P, _I, _P, _I, _I, _I, _P, _P, _P, _P, _D, _D, _D,
                                      _P, _P, _P, _P, _P, _P, _P]
    L.orc_render_occluded.restype = None
    L.orc_render_tiles.argtypes = [_I64, _P, _P, _P, _P, _P, _I, _P, _I, _I, _I, _P, _P, _I, _P, _D, _D, _D,
                                   _P, _P, _P, _P, _P, _P, _P, _P, _P]
    L.orc_render_tiles.restype = None
    L.orc_bin.argtypes = [_I64, _I, _I, _I, _I, _P, _P, _P, _P, _I64, _P, _P, _P]
    L.orc_bin.restype = _I64
    L.orc_render_fwd.argtypes = [_I64, _P, _P, _P, _P, _P, _I, _P, _I, _I, _I, _P, _P, _D, _D, _D,
                                 _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]
    L.orc_render_fwd.restype = _I64
    L.orc_pixel_trace.argtypes = [_I64, _P, _P, _P, _P, _P, _P, _I, _I, _I, _P, _P, _I, _I, _I, _I,
                                  _P, _P, _P, _P]
    L.orc_pixel_trace.restype = _I
    L.orc_render_bwd.argtypes = [_I64, _P, _P, _P, _P, _P, _I, _P, _I, _I, _I, _P, _P, _P, _P, _P,
                                 _P, _P, _P, _P, _P]
    L.orc_render_bwd.restype = None
    L.orc_project_bwd.argtypes = [_I64, _P, _P, _P, _P, _P, _I, _P, _I, _I, _P, _P, _P, _P, _P,
                                  _P, _P, _P, _P, _P, _P]
    L.orc_project_bwd.restype = None
    L.orc_loss_l1.argtypes = [_P, _P, _P, _P, _I, _I, _I, _D, _P, _P]
    L.orc_loss_l1.restype = _D


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


# ----------------------------------------------------------------------------- primitives

def expdet(x) -> np.ndarray:
    x = _c(x, np.float32)
    y = np.empty_like(x)
    lib().orc_expdet_f32(_ptr(x), _ptr(y), x.size)
    return y


def logdet(x) -> np.ndarray:
    x = _c(x, np.float32)
    y = np.empty_like(x)
    lib().orc_logdet_f32(_ptr(x), _ptr(y), x.size)
    return y


@dataclass
class Mirror:
    depth_bits: np.ndarray  # [K*N] uint32
    radius: np.ndarray      # [K*N] int32
    rect: np.ndarray        # [K*N, 4] int32 x0, x1, y0, y1
    count: np.ndarray       # [K*N] uint32 tiles emitted
    uv: np.ndarray          # [K*N, 2] float32
    ell: np.ndarray         # [K*N, 8] float32 widened ellipse: u, v, b, 1/c, sqrt(det), hx, hy, kxy


def project_mirror(means, log_scales, quats, logits, cams, W, H, tile=TILE, near=NEAR) -> Mirror:
    """FP32 discrete mirror of the projection (depth keys, culls, radius, tile rect, and the
    tiles of the rect that the widened alpha >= 1/255 ellipse meets)."""
    means = _c(means, np.float32)
    log_scales = _c(log_scales, np.float32)
    quats = _c(quats, np.float32)
    logits = _c(np.asarray(logits).reshape(-1), np.float32)
    cams = _c(cams, np.float32).reshape(-1, 16)
    N, K = means.shape[0], cams.shape[0]
    out = Mirror(np.empty(K * N, np.uint32), np.empty(K * N, np.int32), np.empty((K * N, 4), np.int32),
                 np.empty(K * N, np.uint32), np.empty((K * N, 2), np.float32), np.empty((K * N, 8), np.float32))
    lib().orc_project_mirror(N, _ptr(means), _ptr(log_scales), _ptr(quats), _ptr(logits), K, _ptr(cams), W, H,
                             tile, near, _ptr(out.depth_bits), _ptr(out.radius), _ptr(out.rect), _ptr(out.count),
                             _ptr(out.uv), _ptr(out.ell))
    return out


def project64(params, cams, W, H) -> np.ndarray:
    """FP64 projection of every (view, Gaussian): [K*N, 8] = u, v, A, B, C, z, opacity, det."""
    means, ls, qs, lg, rgb = params64(*params)
    cams = _c(np.asarray(cams, np.float64), np.float64).reshape(-1, 16)
    N, K = means.shape[0], cams.shape[0]
    out = np.empty((K * N, 8))
    lib().orc_project64(N, _ptr(means), _ptr(ls), _ptr(qs), _ptr(lg), _ptr(rgb), K, _ptr(cams), W, H, _ptr(out))
    return out


def bin_pairs(m: Mirror, N, K, W, H, tile=TILE):
    """Emission + stable sort + tile ranges. Returns (keys u64[P], vals u32[P], ranges u32[K*T,2])."""
    P = int(m.count.astype(np.int64).sum())
    Tx, Ty = -(-W // tile), -(-H // tile)
    keys = np.empty(P, np.uint64)
    vals = np.empty(P, np.uint32)
    ranges = np.empty((K * Tx * Ty, 2), np.uint32)
    got = lib().orc_bin(N, K, W, H, tile, _ptr(m.count), _ptr(m.rect), _ptr(m.ell), _ptr(m.depth_bits), P,
                        _ptr(keys), _ptr(vals), _ptr(ranges))
    assert got == P
    return keys, vals, ranges


def params64(means, log_scales, quats, logits, rgb):
    return tuple(_c(np.asarray(a, np.float64), np.float64) for a in (means, log_scales, quats, logits, rgb))


def render_fwd(params, cams, W, H, vals, ranges, tile=TILE, guard=(GUARD_ALPHA, GUARD_T, GUARD_POWER)):
    means, ls, qs, lg, rgb = params64(*params)
    cams = _c(np.asarray(cams, np.float64), np.float64).reshape(-1, 16)
    N, K = means.shape[0], cams.shape[0]
    vals = _c(vals, np.uint32)
    ranges = _c(ranges, np.uint32)
    o = {
        "rgb": np.empty((K, 3, H, W)), "depth": np.empty((K, H, W)), "T": np.empty((K, H, W)),
        "last": np.empty((K, H, W), np.int32), "evals": np.empty((K, H, W), np.int32),
        "near": np.empty((K, H, W), np.int32), "alt_rgb": np.empty((K, 3, H, W)),
        "alt_depth": np.empty((K, H, W)), "alt_T": np.empty((K, H, W)), "alt_last": np.empty((K, H, W), np.int32),
    }
    total = lib().orc_render_fwd(N, _ptr(means), _ptr(ls), _ptr(qs), _ptr(lg), _ptr(rgb), K, _ptr(cams), W, H,
                                 tile, _ptr(vals), _ptr(ranges), guard[0], guard[1], guard[2], _ptr(o["rgb"]),
                                 _ptr(o["depth"]), _ptr(o["T"]), _ptr(o["last"]), _ptr(o["evals"]),
                                 _ptr(o["near"]), _ptr(o["alt_rgb"]), _ptr(o["alt_depth"]), _ptr(o["alt_T"]),
                                 _ptr(o["alt_last"]))
    o["total_evals"] = int(total)
    return o


def render_occluded(params, cams, W, H, vals, ranges, ext_depth, ext_rgb=None, tile=TILE,
                    guard=(GUARD_ALPHA, GUARD_T, GUARD_POWER)):
    """FP64 render occluded by an external surface (depth [K,H,W], colour [K,3,H,W] or None)."""
    means, ls, qs, lg, rgb = params64(*params)
    cams = _c(np.asarray(cams, np.float64), np.float64).reshape(-1, 16)
    N, K = means.shape[0], cams.shape[0]
    ed = _c(ext_depth, np.float32)
    er = _c(ext_rgb, np.float32) if ext_rgb is not None else None
    o = {"rgb": np.empty((K, 3, H, W)), "depth": np.empty((K, H, W)), "T": np.empty((K, H, W)),
         "near": np.empty((K, H, W), np.int32), "alt_rgb": np.empty((K, 3, H, W)), "alt_depth": np.empty((K, H, W)),
         "alt_T": np.empty((K, H, W))}
    lib().orc_render_occluded(N, _ptr(means), _ptr(ls), _ptr(qs), _ptr(lg), _ptr(rgb), K, _ptr(cams), W, H, tile,
                              _ptr(_c(vals, np.uint32)), _ptr(_c(ranges, np.uint32)), _ptr(ed),
                              _ptr(er) if er is not None else None, *guard, _ptr(o["rgb"]), _ptr(o["depth"]),
                              _ptr(o["T"]), _ptr(o["near"]), _ptr(o["alt_rgb"]), _ptr(o["alt_depth"]),
                              _ptr(o["alt_T"]))
    return o


def render_tiles(params, cams, W, H, vals, ranges, tiles, tile=TILE,
                 guard=(GUARD_ALPHA, GUARD_T, GUARD_POWER)):
    """FP64 render of the listed global tiles only (every pixel of each), with the same
    compositing and guard-band outputs as render_fwd. Returns arrays [n, 16, 16] (rgb
    [n, 3, 16, 16]); near = -1 marks pixels outside the image."""
    means, ls, qs, lg, rgb = params64(*params)
    cams = _c(np.asarray(cams, np.float64), np.float64).reshape(-1, 16)
    N = means.shape[0]
    tl = _c(np.asarray(tiles, np.int64), np.int64)
    n, P = len(tl), tile * tile
    o = {"rgb": np.empty((n, 3, P)), "depth": np.empty((n, P)), "T": np.empty((n, P)),
         "last": np.empty((n, P), np.int32), "near": np.empty((n, P), np.int32), "alt_rgb": np.empty((n, 3, P)),
         "alt_depth": np.empty((n, P)), "alt_T": np.empty((n, P)), "alt_last": np.empty((n, P), np.int32)}
    lib().orc_render_tiles(N, _ptr(means), _ptr(ls), _ptr(qs), _ptr(lg), _ptr(rgb), cams.shape[0], _ptr(cams), W, H,
                           tile, _ptr(_c(vals, np.uint32)), _ptr(_c(ranges, np.uint32)), n, _ptr(tl), *guard,
                           _ptr(o["rgb"]), _ptr(o["depth"]), _ptr(o["T"]), _ptr(o["last"]), _ptr(o["near"]),
                           _ptr(o["alt_rgb"]), _ptr(o["alt_depth"]), _ptr(o["alt_T"]), _ptr(o["alt_last"]))
    return {k: (v.reshape(n, 3, tile, tile) if v.ndim == 3 else v.reshape(n, tile, tile)) for k, v in o.items()}


def pixel_trace(params, cam, W, H, vals, ranges, k, px, py, tile=TILE, max_n=4096):
    means, ls, qs, lg, rgb = params64(*params)
    cam = _c(np.asarray(cam, np.float64).reshape(16), np.float64)
    g = np.empty(max_n, np.int32)
    a = np.empty(max_n)
    T = np.empty(max_n)
    Tf = np.empty(1)
    n = lib().orc_pixel_trace(means.shape[0], _ptr(means), _ptr(ls), _ptr(qs), _ptr(lg), _ptr(rgb), _ptr(cam), W,
                              H, tile, _ptr(_c(vals, np.uint32)), _ptr(_c(ranges, np.uint32)), k, px, py, max_n,
                              _ptr(g), _ptr(a), _ptr(T), _ptr(Tf))
    return g[:n].copy(), a[:n].copy(), T[:n].copy(), float(Tf[0])


def render_bwd(params, cams, W, H, vals, ranges, dL_drgb, dL_ddepth, dL_dT=None, tile=TILE):
    means, ls, qs, lg, rgb = params64(*params)
    cams = _c(np.asarray(cams, np.float64), np.float64).reshape(-1, 16)
    N, K = means.shape[0], cams.shape[0]
    gr = _c(np.asarray(dL_drgb, np.float64), np.float64)
    gd = _c(np.asarray(dL_ddepth, np.float64), np.float64)
    gt = None if dL_dT is None else _c(np.asarray(dL_dT, np.float64), np.float64)
    o = {"d_uv": np.empty((K * N, 2)), "d_conic": np.empty((K * N, 3)), "d_z": np.empty(K * N),
         "d_opac": np.empty(N), "d_rgb": np.empty((N, 3))}
    lib().orc_render_bwd(N, _ptr(means), _ptr(ls), _ptr(qs), _ptr(lg), _ptr(rgb), K, _ptr(cams), W, H, tile,
                         _ptr(_c(vals, np.uint32)), _ptr(_c(ranges, np.uint32)), _ptr(gr), _ptr(gd),
                         None if gt is None else _ptr(gt), _ptr(o["d_uv"]), _ptr(o["d_conic"]), _ptr(o["d_z"]),
                         _ptr(o["d_opac"]), _ptr(o["d_rgb"]))
    return o


def project_bwd(params, cams, W, H, g2d):
    means, ls, qs, lg, rgb = params64(*params)
    cams = _c(np.asarray(cams, np.float64), np.float64).reshape(-1, 16)
    N, K = means.shape[0], cams.shape[0]
    o = {"means": np.empty((N, 3)), "log_scales": np.empty((N, 3)), "quats": np.empty((N, 4)),
         "opacity_logits": np.empty(N), "rgb": np.empty((N, 3)), "pose": np.empty((K, 6))}
    d = {k: _c(g2d[k], np.float64) for k in ("d_uv", "d_conic", "d_z", "d_opac", "d_rgb")}
    lib().orc_project_bwd(N, _ptr(means), _ptr(ls), _ptr(qs), _ptr(lg), _ptr(rgb), K, _ptr(cams), W, H,
                          _ptr(d["d_uv"]), _ptr(d["d_conic"]), _ptr(d["d_z"]), _ptr(d["d_opac"]),
                          _ptr(d["d_rgb"]), _ptr(o["means"]), _ptr(o["log_scales"]), _ptr(o["quats"]),
                          _ptr(o["opacity_logits"]), _ptr(o["rgb"]), _ptr(o["pose"]))
    return o


def loss_l1(rgb, depth, rgb_t, depth_t, lambda_depth=0.1):
    rgb = _c(np.asarray(rgb, np.float64), np.float64)
    depth = _c(np.asarray(depth, np.float64), np.float64)
    rgb_t = _c(np.asarray(rgb_t, np.float64), np.float64)
    depth_t = _c(np.asarray(depth_t, np.float64), np.float64)
    K, _, H, W = rgb.shape
    gr = np.empty_like(rgb)
    gd = np.empty_like(depth)
    L = lib().orc_loss_l1(_ptr(rgb), _ptr(depth), _ptr(rgb_t), _ptr(depth_t), K, H, W, lambda_depth,
                          _ptr(gr), _ptr(gd))
    return float(L), gr, gd


# ----------------------------------------------------------------------------- pipelines

@dataclass
class Lists:
    mirror: Mirror
    keys: np.ndarray
    vals: np.ndarray
    ranges: np.ndarray


def discrete(params, cams, W, H, tile=TILE, near=NEAR) -> Lists:
    """Mirror + binning for float32-stored parameters."""
    means, ls, qs, lg = params[0], params[1], params[2], params[3]
    cams = np.asarray(cams, np.float32).reshape(-1, 16)
    m = project_mirror(means, ls, qs, lg, cams, W, H, tile, near)
    keys, vals, ranges = bin_pairs(m, np.asarray(means).shape[0], cams.shape[0], W, H, tile)
    return Lists(m, keys, vals, ranges)


def forward(params, cams, W, H, tile=TILE, guard=(GUARD_ALPHA, GUARD_T, GUARD_POWER)):
    """Full oracle forward: discrete lists from the FP32 mirror, FP64 compositing."""
    lists = discrete(params, cams, W, H, tile)
    out = render_fwd(params, cams, W, H, lists.vals, lists.ranges, tile, guard)
    out["lists"] = lists
    return out


def backward(params, cams, W, H, lists: Lists, dL_drgb, dL_ddepth, dL_dT=None, tile=TILE):
    """Full oracle backward: screen-space gradients, then parameter and pose gradients."""
    g2 = render_bwd(params, cams, W, H, lists.vals, lists.ranges, dL_drgb, dL_ddepth, dL_dT, tile)
    g = project_bwd(params, cams, W, H, g2)
    g["screen"] = g2
    return g
