"""Host-side checks of the C ABI (no GPU): the library loads, exports every entry
point declared in include/gs.h, and its host-only calls (workspace sizing and
layout, argument validation) behave as documented."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_06433_gb300 import build
    from paper_2509_06433_gb300 import _lib
    build()
    return _lib.load()


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    return re.findall(r"GS_API\s+gs_status_t\s+(\w+)\s*\(", src)


def test_header_declares_the_hot_path():
    names = declared_entry_points()
    for n in ("gs_project", "gs_bin_sort", "gs_raster_fwd", "gs_raster_bwd", "gs_project_bwd"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2509_06433_gb300._lib import EXPORTS
    names = declared_entry_points()
    assert set(names) == set(EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_debug_build_exports_the_same_entry_points():
    # the index-checking build (GS_DEBUG) is a drop-in replacement of the release library
    from paper_2509_06433_gb300.build import build
    path = build(debug=True)
    dbg = ctypes.CDLL(path)
    for n in declared_entry_points():
        assert hasattr(dbg, n), n


def _cfg(W=640, H=480, K=1, N=100_000, cap=1 << 20, tile=16, near=0.2):
    from paper_2509_06433_gb300._lib import GsConfig
    return GsConfig(W, H, tile, K, N, cap, near, 0.1, 0, 0)


def test_workspace_size_and_layout(lib):
    from paper_2509_06433_gb300._lib import GsWsLayout
    cfg = _cfg()
    n = ctypes.c_size_t()
    assert lib.gs_workspace_size(ctypes.byref(cfg), ctypes.byref(n)) == 0
    lay = GsWsLayout()
    assert lib.gs_workspace_layout(ctypes.byref(cfg), ctypes.byref(lay)) == 0
    assert lay.total == n.value
    assert (lay.tiles_x, lay.tiles_y) == (40, 30)
    # 1200 tiles -> 11 tile bits -> 2 pair-sort passes of 8 bits (depth is ordered per item first)
    assert lay.sort_passes == 2
    offs = [lay.status, lay.proj_uv, lay.proj_conic, lay.proj_tiles, lay.proj_depth_key, lay.proj_radius,
            lay.color_opacity, lay.ranges, lay.pair_grads]
    assert all(o % 256 == 0 for o in offs + [lay.keys_sorted, lay.vals_sorted])
    assert len(set(offs)) == len(offs) and max(offs) < lay.total
    # sizes grow with the capacity and the view count
    n2 = ctypes.c_size_t()
    assert lib.gs_workspace_size(ctypes.byref(_cfg(cap=1 << 21)), ctypes.byref(n2)) == 0 and n2.value > n.value
    k8 = GsWsLayout()
    assert lib.gs_workspace_layout(ctypes.byref(_cfg(K=8)), ctypes.byref(k8)) == 0
    assert k8.sort_passes == 2  # 9600 tiles -> 14 bits


@pytest.mark.parametrize("bad", [dict(tile=8), dict(W=0), dict(H=20000), dict(K=0), dict(N=-1), dict(cap=0),
                                 dict(cap=1 << 30), dict(near=0.0)])
def test_invalid_configs_rejected(lib, bad):
    n = ctypes.c_size_t()
    assert lib.gs_workspace_size(ctypes.byref(_cfg(**bad)), ctypes.byref(n)) == 1  # GS_ERR_INVALID_ARG


def test_calls_reject_bad_workspace_before_touching_the_device(lib):
    cfg = _cfg(N=10, cap=1024)
    n = ctypes.c_size_t()
    lib.gs_workspace_size(ctypes.byref(cfg), ctypes.byref(n))
    # null / misaligned workspace -> INVALID_ARG, undersized -> WORKSPACE_TOO_SMALL
    assert lib.gs_bin_sort(ctypes.byref(cfg), None, n.value, None) == 1
    assert lib.gs_bin_sort(ctypes.byref(cfg), ctypes.c_void_p(0x1001), n.value, None) == 1
    assert lib.gs_bin_sort(ctypes.byref(cfg), ctypes.c_void_p(0x1000), n.value - 1, None) == 2
    assert lib.gs_sort_pairs(None, None, -1, 64, None, 0, None, None) == 1
    assert lib.gs_sort_pairs(None, None, 0, 64, None, 0, None, None) == 0  # empty sort is a no-op
    assert lib.gs_sort_pairs(None, None, 10, 65, None, 0, None, None) == 1
