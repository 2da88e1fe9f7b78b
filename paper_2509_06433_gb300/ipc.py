"""A Gaussian map shared between two processes on one GPU (Sec. III, Fig. 5: the map optimiser
and the interactive viewer each own a renderer and read the same map in GPU memory).

``SharedMap`` (optimiser process) keeps the five FP32 Gaussian arrays in one device buffer,
exports it with gs_ipc_export and creates the interprocess "published" event. Its
``descriptor()`` is a small JSON-able dict (hex handles, N, colour width) to hand to the other
process. ``MapView`` (viewer process) imports the buffer and the event; its ``gaussians`` can be
passed to a Rasterizer like api.Gaussians, and ``wait()`` orders the next render after the last
published update (reads may still overlap a later update: see include/gs.h).
"""
from __future__ import annotations

import ctypes

import torch

from . import api
from ._lib import GsGaussians, call

GS_F32 = 0


class IpcMemHandle(ctypes.Structure):
    _fields_ = [("bytes", ctypes.c_uint8 * 128)]


class IpcEventHandle(ctypes.Structure):
    _fields_ = [("bytes", ctypes.c_uint8 * 64)]


def _layout(N: int, color_width: int):
    """(name, offset in floats, shape) of the five arrays in the shared buffer."""
    out, off = [], 0
    for name, w in (("means", 3), ("log_scales", 3), ("quats", 4), ("opacity_logits", 1), ("rgb", color_width)):
        shape = (N,) if w == 1 else (N, w)
        out.append((name, off, shape))
        off += N * w
    return out, off


class SharedMap:
    """Exporter side. ``g`` (api.Gaussians) views the shared buffer; map updates write into it."""

    def __init__(self, N: int, color_width: int = 3, device="cuda"):
        self.N, self.color_width = int(N), int(color_width)
        lay, total = _layout(self.N, self.color_width)
        self.buffer = torch.zeros(total, dtype=torch.float32, device=device)
        views = {name: self.buffer[off:off + int(torch.Size(shape).numel())].view(shape) for name, off, shape in lay}
        self.g = api.Gaussians(views["means"], views["log_scales"], views["quats"], views["opacity_logits"],
                               views["rgb"])
        self._mem = IpcMemHandle()
        call("gs_ipc_export", ctypes.c_void_p(self.buffer.data_ptr()), ctypes.c_size_t(total * 4),
             ctypes.byref(self._mem))
        self._event = ctypes.c_void_p()
        self._evh = IpcEventHandle()
        call("gs_ipc_event_create", ctypes.byref(self._event), ctypes.byref(self._evh))

    def load(self, g: "api.Gaussians"):
        """Copies a map into the shared buffer (FP32)."""
        for name in ("means", "log_scales", "quats", "opacity_logits", "rgb"):
            getattr(self.g, name).copy_(getattr(g, name).reshape(getattr(self.g, name).shape))

    def publish(self, stream=None):
        """Records the published event after the updates enqueued so far on `stream`."""
        s = stream if stream is not None else torch.cuda.current_stream()
        call("gs_ipc_event_record", self._event, ctypes.c_void_p(s.cuda_stream))

    def descriptor(self) -> dict:
        return {"mem": bytes(self._mem.bytes).hex(), "event": bytes(self._evh.bytes).hex(), "N": self.N,
                "color_width": self.color_width}

    def close(self):
        if self._event:
            call("gs_ipc_event_destroy", self._event)
            self._event = ctypes.c_void_p()


class _RawGaussians:
    """Device pointers of a map this process does not own (duck-types api.Gaussians for the
    rasterizer: N and struct())."""

    def __init__(self, ptrs: dict, N: int):
        self.ptrs, self._N = ptrs, N

    @property
    def N(self) -> int:
        return self._N

    def struct(self) -> GsGaussians:
        p = self.ptrs
        return GsGaussians(p["means"], p["log_scales"], p["quats"], p["opacity_logits"], p["rgb"], GS_F32, GS_F32)


class MapView:
    """Importer side (another process on the same GPU)."""

    def __init__(self, desc: dict):
        self.N, self.color_width = int(desc["N"]), int(desc["color_width"])
        mem = IpcMemHandle()
        ctypes.memmove(mem.bytes, bytes.fromhex(desc["mem"]), 128)
        evh = IpcEventHandle()
        ctypes.memmove(evh.bytes, bytes.fromhex(desc["event"]), 64)
        self._ptr = ctypes.c_void_p()
        size = ctypes.c_size_t()
        call("gs_ipc_import", ctypes.byref(mem), ctypes.byref(self._ptr), ctypes.byref(size))
        lay, total = _layout(self.N, self.color_width)
        if size.value != total * 4:
            raise ValueError(f"shared map holds {size.value} bytes, the descriptor says {total * 4}")
        base = self._ptr.value
        self.gaussians = _RawGaussians({name: ctypes.c_void_p(base + 4 * off) for name, off, _ in lay}, self.N)
        self._event = ctypes.c_void_p()
        call("gs_ipc_event_open", ctypes.byref(evh), ctypes.byref(self._event))

    def wait(self, stream=None):
        """The next work enqueued on `stream` starts after the last published update."""
        s = stream if stream is not None else torch.cuda.current_stream()
        call("gs_ipc_stream_wait", ctypes.c_void_p(s.cuda_stream), self._event)

    def close(self):
        if self._event:
            call("gs_ipc_event_destroy", self._event)
            self._event = ctypes.c_void_p()
        if self._ptr:
            call("gs_ipc_release", self._ptr)
            self._ptr = ctypes.c_void_p()
