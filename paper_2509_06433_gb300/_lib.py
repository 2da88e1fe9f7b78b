"""ctypes binding of ``libgs.so`` (the C ABI in ``include/gs.h``).

Argument marshalling only: every step of the rasterizer runs in the library's
sm_103a kernels. Tensors are torch CUDA tensors; streams default to torch's
current stream. If the library has not been built, loading fails loudly; there
is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB, LIB_DEBUG

c_int32, c_int64, c_float, c_void_p, c_size_t, c_uint32 = (ctypes.c_int32, ctypes.c_int64, ctypes.c_float,
                                                          ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32)

GS_OK = 0
STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_WORKSPACE_TOO_SMALL", 3: "GS_ERR_CAPACITY_OVERFLOW",
                4: "GS_ERR_DEVICE_TIMEOUT", 5: "GS_ERR_CUDA", 6: "GS_ERR_NONFINITE", 7: "GS_ERR_SIZE_LIMIT",
                8: "GS_ERR_INDEX_CHECK"}
SORT_NOALLOC_MAX_PAIRS = 1048576
DEVERR_PAIR_OVERFLOW, DEVERR_TIMEOUT, DEVERR_NONFINITE = 0x1, 0x2, 0x4
GS_F32, GS_BF16, GS_F16 = 0, 1, 2

#: every entry point declared in include/gs.h
EXPORTS = ("gs_workspace_size", "gs_workspace_layout", "gs_read_status", "gs_project", "gs_bin_sort",
           "gs_raster_fwd", "gs_raster_fwd_stats", "gs_raster_fwd_l1", "gs_raster_fwd_l1_bwd", "gs_raster_fwd_occluded", "gs_loss_l1", "gs_raster_bwd", "gs_project_bwd", "gs_screen_grads",
           "gs_pose_adam_step", "gs_sort_pairs_tmp_size", "gs_sort_pairs", "gs_sort_diag_withheld_tile",
           "gs_sort_pairs_noalloc", "gs_map_adam_state_size", "gs_map_adam_step", "gs_keyframe_tmp_size",
           "gs_keyframe_insert", "gs_metrics_tmp_size", "gs_psnr", "gs_ssim",
           "gs_ipc_export", "gs_ipc_import", "gs_ipc_release", "gs_ipc_event_create", "gs_ipc_event_open",
           "gs_ipc_event_record", "gs_ipc_stream_wait", "gs_ipc_event_destroy")


class GsConfig(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("tile", c_int32), ("num_views", c_int32),
                ("num_gaussians", c_int64), ("pair_capacity", c_int64), ("near_plane", c_float),
                ("lambda_depth", c_float), ("fwd_px_per_thread", c_int32), ("bwd_px_per_thread", c_int32),
                ("fwd_chunk", c_int32), ("bwd_chunk", c_int32), ("color_mode", c_int32), ("sh_degree", c_int32),
                ("raster_blocks_per_sm", c_int32)]


class GsGaussians(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("log_scales", c_void_p), ("quats", c_void_p), ("opacity_logits", c_void_p),
                ("rgb", c_void_p), ("dtype", ctypes.c_int), ("means_dtype", ctypes.c_int)]


class GsGrads(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("log_scales", c_void_p), ("quats", c_void_p), ("opacity_logits", c_void_p),
                ("rgb", c_void_p), ("pose", c_void_p), ("overwrite", c_int32)]


class GsAdam(ctypes.Structure):
    _fields_ = [("lr_means", c_float), ("lr_log_scales", c_float), ("lr_quats", c_float), ("lr_opacity", c_float),
                ("lr_rgb", c_float), ("beta1", c_float), ("beta2", c_float), ("eps", c_float),
                ("color_width", c_int32)]


class GsWsLayout(ctypes.Structure):
    _fields_ = [("total", c_size_t), ("status", c_size_t), ("proj_uv", c_size_t), ("proj_conic", c_size_t),
                ("proj_tiles", c_size_t), ("proj_depth_key", c_size_t), ("proj_radius", c_size_t),
                ("color_opacity", c_size_t), ("keys_sorted", c_size_t), ("vals_sorted", c_size_t),
                ("ranges", c_size_t), ("pair_grads", c_size_t), ("sort_passes", c_int32), ("tiles_x", c_int32),
                ("tiles_y", c_int32), ("bin_sort_launches", c_int32),
                ("pair_valid", c_size_t), ("live_mask", c_size_t), ("project_launches", c_int32),
                ("project_bwd_launches", c_int32), ("live_off", c_size_t)]


class GsError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} returned {STATUS_NAMES.get(code, code)}")
        self.code = code


_lock = threading.Lock()
_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load the built library (``build()`` first). Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or (LIB_DEBUG if os.environ.get("GS_DEBUG") == "1" else LIB)
            if not os.path.exists(p):
                raise RuntimeError(f"CUDA library not built ({p}); run paper_2509_06433_gb300.build.build()")
            L = ctypes.CDLL(p)
            P = c_void_p
            sig = {
                "gs_workspace_size": [P, P],
                "gs_workspace_layout": [P, P],
                "gs_read_status": [P, P, c_size_t, P, P, P, P],
                "gs_project": [P, P, P, P, c_size_t, P],
                "gs_bin_sort": [P, P, c_size_t, P],
                "gs_raster_fwd": [P, P, c_size_t, P, P, P, P, P],
                "gs_raster_fwd_stats": [P, P, c_size_t, P, P, P, P, P],
                "gs_raster_fwd_l1": [P, P, c_size_t, P, P, P, P, P, P, P, P, P, P],
                "gs_raster_fwd_l1_bwd": [P, P, c_size_t, P, P, P, P, P, P, P, P, P, P],
                "gs_raster_fwd_occluded": [P, P, c_size_t, P, P, P, P, P, P, P],
                "gs_loss_l1": [P, P, P, P, P, P, P, P, P, c_size_t, P],
                "gs_raster_bwd": [P, P, c_size_t, P, P, P, P, P, P, P, P],
                "gs_project_bwd": [P, P, P, P, c_size_t, P, P],
                "gs_screen_grads": [P, P, c_size_t, P, P, P, P, P, P],
                "gs_sort_pairs_tmp_size": [c_int64, P],
                "gs_sort_pairs": [P, P, c_int64, c_int32, P, c_size_t, P, P],
                "gs_sort_pairs_noalloc": [P, P, c_int64, c_int32, P, P],
                "gs_map_adam_state_size": [c_int64, c_int32, P],
                "gs_map_adam_step": [c_int64, P, P, P, P, P, P, P, P, P, P],
                "gs_keyframe_tmp_size": [c_int32, c_int32, c_int32, P],
                "gs_keyframe_insert": [P, P, P, P, c_int32, c_int32, c_int32, c_float, c_float, c_float, c_float,
                                       P, P, P, P, P, c_int64, c_int64, P, P, c_size_t, P],
                "gs_metrics_tmp_size": [c_int32, c_int32, c_int32, c_int32, P],
                "gs_psnr": [P, P, c_int32, c_int32, c_int32, c_int32, c_float, P, P, c_size_t, P],
                "gs_ssim": [P, P, c_int32, c_int32, c_int32, c_int32, c_float, P, P, P, c_size_t, P],
                "gs_ipc_export": [P, c_size_t, P],
                "gs_ipc_import": [P, P, P],
                "gs_ipc_release": [P],
                "gs_ipc_event_create": [P, P],
                "gs_ipc_event_open": [P, P],
                "gs_ipc_event_record": [P, P],
                "gs_ipc_stream_wait": [P, P],
                "gs_ipc_event_destroy": [P],
                "gs_sort_diag_withheld_tile": [P, P, c_int64, P, c_size_t, P, P],
                "gs_pose_adam_step": [P, P, P, c_int32, c_float, c_float, c_float, c_float, c_float, c_int32, P],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            _lib = L
    return _lib


def call(name, *args):
    code = getattr(load(), name)(*args)
    if code != GS_OK:
        raise GsError(name, code)
    return code
