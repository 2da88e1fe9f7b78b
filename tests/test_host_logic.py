"""Host-side choices of the mapping step (CPU only)."""
import types

from paper_2509_06433_gb300 import api
from paper_2509_06433_gb300.tracking import fuses_backward


def _r(fpx, bpx, **attrs):
    cfg = api.make_config(640, 480, 1, 1000, 1 << 16, fwd_px=fpx, bwd_px=bpx)
    return types.SimpleNamespace(cfg=cfg, **attrs)


def test_one_launch_only_with_one_pixels_per_thread_value():
    assert fuses_backward(_r(0, 0)) and fuses_backward(_r(4, 4)) and fuses_backward(_r(2, 0))  # 0 = default 2
    assert not fuses_backward(_r(4, 2)) and not fuses_backward(_r(1, 0))


def test_autotuned_choice_is_respected():
    assert fuses_backward(_r(4, 4, fused_compositing=True))
    assert not fuses_backward(_r(4, 4, fused_compositing=False))
    assert not fuses_backward(_r(4, 2, fused_compositing=True))  # never across two variants
