"""Binary dump and load of a Gaussian map (with optional camera poses and mapping-optimiser
state), for reproducible runs and for resuming a mapping session.

The file is a numpy .npz archive: the five attribute arrays under their names, each in its
storage dtype (float32, or bfloat16 / float16 kept bit for bit as 16-bit words), plus ``cams``
[K, 16] and the optimiser's ``adam_state`` when given, and a small ``meta`` record (format
version, dtypes, N, the SH degree when the colour holds spherical-harmonic coefficients).
Loading restores every array bit for bit.
"""
from __future__ import annotations

import json

import numpy as np
import torch

from . import api

FORMAT = 1
_NAMES = ("means", "log_scales", "quats", "opacity_logits", "rgb")
_BITS16 = {torch.bfloat16: "bfloat16", torch.float16: "float16"}
_FROM16 = {v: k for k, v in _BITS16.items()}


def _to_numpy(t: torch.Tensor):
    t = t.detach().contiguous().cpu()
    if t.dtype in _BITS16:
        return t.view(torch.int16).numpy(), _BITS16[t.dtype]
    return t.numpy(), str(t.dtype).replace("torch.", "")


def _from_numpy(a: np.ndarray, dtype: str, device) -> torch.Tensor:
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype in _FROM16:
        t = t.view(_FROM16[dtype])
    return t.to(device)


def save(path: str, g: "api.Gaussians", cams: torch.Tensor = None, optimizer: "api.MapOptimizer" = None,
         sh_degree: int = None):
    """Writes the map (and the cameras / optimiser state when given) to `path` (.npz)."""
    arrays, dtypes = {}, {}
    for name in _NAMES:
        arrays[name], dtypes[name] = _to_numpy(getattr(g, name))
    if cams is not None:
        arrays["cams"], dtypes["cams"] = _to_numpy(cams)
    if optimizer is not None:
        arrays["adam_state"], dtypes["adam_state"] = _to_numpy(optimizer.state)
        for name in _NAMES:  # the FP32 masters, when the map itself is stored in reduced precision
            if optimizer.storage is not None:
                arrays["master_" + name], dtypes["master_" + name] = _to_numpy(getattr(optimizer.masters, name))
    meta = {"format": FORMAT, "N": g.N, "dtypes": dtypes, "sh_degree": sh_degree}
    np.savez(path, meta=np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8), **arrays)


def load(path: str, device="cuda"):
    """Returns (gaussians, cams or None, extras) with extras = {"adam_state", "masters", "sh_degree"}
    (None where absent); every array on `device`, in its stored dtype, bit for bit."""
    with np.load(path) as z:
        meta = json.loads(bytes(z["meta"]).decode())
        if meta.get("format") != FORMAT:
            raise ValueError(f"unsupported map file format {meta.get('format')}")
        dt = meta["dtypes"]
        g = api.Gaussians(*(_from_numpy(z[n], dt[n], device) for n in _NAMES))
        cams = _from_numpy(z["cams"], dt["cams"], device) if "cams" in z.files else None
        state = _from_numpy(z["adam_state"], dt["adam_state"], device) if "adam_state" in z.files else None
        masters = None
        if "master_means" in z.files:
            masters = api.Gaussians(*(_from_numpy(z["master_" + n], dt["master_" + n], device) for n in _NAMES))
    return g, cams, {"adam_state": state, "masters": masters, "sh_degree": meta.get("sh_degree")}


def restore_optimizer(optimizer: "api.MapOptimizer", extras: dict):
    """Copies a loaded optimiser state (and FP32 masters) into `optimizer`, built on the loaded map."""
    if extras.get("adam_state") is not None:
        optimizer.state.copy_(extras["adam_state"])
    if extras.get("masters") is not None and optimizer.storage is not None:
        for name in _NAMES:
            getattr(optimizer.masters, name).copy_(getattr(extras["masters"], name))
