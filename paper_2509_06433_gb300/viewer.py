"""Interactive-viewer process: renders a Gaussian map shared by another process (the map
optimiser) over CUDA IPC, from viewer poses, into headless device buffers (Sec. III: the viewer
has its own renderer and reads the map in GPU memory; it renders several viewpoints at once
for a VR headset, at the paper's 672 x 376).

Run as ``python -m paper_2509_06433_gb300.viewer --desc map.json --out result.json`` where
map.json is ``ipc.SharedMap.descriptor()``. Each frame waits on the map's published event,
renders all viewpoints (one K-view launch per stage) and synchronises, as a viewer that
presents every frame would. The poses orbit a target point (a stereo pair of eyes 64 mm apart
per viewpoint pair) unless explicit cameras are given (--cams, a float32 .npy [views, 16]).
The result file holds the frame rate; --save writes the last frame (rgb, depth, T, last) as
.npz. With --control, frames are rendered only while that file exists (the viewer idles,
polling every millisecond, otherwise) and the loop runs until the --stop file appears; the
frame rate then counts the frames and the time spent while active.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np


def orbit_camera(target, radius, yaw, pitch, f, W, H, up=(0.0, -1.0, 0.0), eye_offset=0.0):
    """Camera (16 floats: fx fy cx cy, R row-major, t; world -> camera, x right, y down, z
    forward) on a sphere around `target`, looking at it; eye_offset shifts it along its x axis."""
    target = np.asarray(target, np.float64)
    up = np.asarray(up, np.float64)
    # position: yaw about the up axis, pitch towards it, starting behind the target along -z
    back = np.array([math.sin(yaw) * math.cos(pitch), 0.0, -math.cos(yaw) * math.cos(pitch)])
    c = target + radius * back + up * (radius * math.sin(pitch))
    z = target - c
    z /= np.linalg.norm(z)
    x = np.cross(-up, z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    c = c + eye_offset * x
    R = np.stack([x, y, z])
    t = -R @ c
    return np.concatenate([[f, f, W / 2.0, H / 2.0], R.reshape(-1), t]).astype(np.float32)


def orbit_rig(i, views, target, radius, f, W, H, sweep_deg=30.0, period=240):
    """The viewpoints of frame i: pairs of eyes 64 mm apart, pair p offset by 10 deg of yaw."""
    yaw0 = math.radians(sweep_deg) * math.sin(2 * math.pi * i / period)
    cams = []
    for v in range(views):
        pair, eye = divmod(v, 2)
        cams.append(orbit_camera(target, radius, yaw0 + math.radians(10.0) * pair, math.radians(10.0), f, W, H,
                                 eye_offset=(eye - 0.5) * 0.064 if views > 1 else 0.0))
    return np.stack(cams)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--desc", required=True, help="JSON descriptor of the shared map (ipc.SharedMap.descriptor)")
    ap.add_argument("--out", required=True, help="result JSON written at the end")
    ap.add_argument("--ready", default=None, help="file created once the viewer is warmed up")
    ap.add_argument("--width", type=int, default=672)
    ap.add_argument("--height", type=int, default=376)
    ap.add_argument("--views", type=int, default=2)
    ap.add_argument("--frames", type=int, default=300)
    ap.add_argument("--f", type=float, default=336.0)
    ap.add_argument("--target", type=float, nargs=3, default=(0.0, 0.0, 5.0))
    ap.add_argument("--radius", type=float, default=4.0)
    ap.add_argument("--cams", default=None, help="float32 .npy [views, 16]: fixed cameras instead of the orbit")
    ap.add_argument("--save", default=None, help=".npz path for the last frame (rgb, depth, T, last)")
    ap.add_argument("--control", default=None, help="render only while this file exists (until --stop)")
    ap.add_argument("--stop", default=None, help="with --control: end when this file exists")
    a = ap.parse_args(argv)

    import torch

    from . import api
    from .build import build
    from .ipc import MapView
    build()
    with open(a.desc) as fh:
        desc = json.load(fh)
    view = MapView(desc)
    W, H = a.width, a.height
    fixed = np.load(a.cams).astype(np.float32).reshape(-1, 16) if a.cams else None
    K = fixed.shape[0] if fixed is not None else a.views
    rig = (lambda i: fixed) if fixed is not None else (  # noqa: E731
        lambda i: orbit_rig(i, K, a.target, a.radius, a.f, W, H))
    host = torch.empty((K, 16), dtype=torch.float32).pin_memory()
    cams = torch.empty((K, 16), dtype=torch.float32, device="cuda")
    r = api.Rasterizer(W, H, K, view.N, pair_capacity=max(1 << 20, 4 * view.N * K))
    out = r.new_outputs()  # the headless frame buffers

    def frame(i):
        host.copy_(torch.from_numpy(rig(i)))
        cams.copy_(host, non_blocking=True)
        view.wait()
        r.render(view.gaussians, cams, out)

    view.wait()
    r.plan(view.gaussians, torch.from_numpy(rig(0)).cuda(), headroom=2.0)
    for i in range(3):
        frame(i)
    torch.cuda.synchronize()
    if a.ready:
        open(a.ready, "w").close()
    frame_ms = []
    i = 0
    if a.control:  # render while the control file exists, until the stop file appears
        while not (a.stop and os.path.exists(a.stop)):
            if not os.path.exists(a.control):
                time.sleep(1e-3)
                continue
            s = time.perf_counter()
            frame(i)
            torch.cuda.current_stream().synchronize()  # a viewer presents every frame
            frame_ms.append(1e3 * (time.perf_counter() - s))
            i += 1
        n, dt = len(frame_ms), 1e-3 * sum(frame_ms)
    else:
        t0 = time.perf_counter()
        for i in range(a.frames):
            s = time.perf_counter()
            frame(i)
            torch.cuda.current_stream().synchronize()  # a viewer presents every frame
            frame_ms.append(1e3 * (time.perf_counter() - s))
        n, dt = a.frames, time.perf_counter() - t0
    _, err, total, _ = r.status()
    if a.save:
        np.savez(a.save, **{k: v.cpu().numpy() for k, v in out.items()})
    res = {"fps": n / dt if dt > 0 else 0.0, "frames": n, "seconds": dt, "views": K, "width": W, "height": H,
           "frame_ms_median": float(np.median(frame_ms)) if frame_ms else None,
           "frame_ms_p99": float(np.percentile(frame_ms, 99)) if frame_ms else None,
           "pairs_last_frame": int(total), "device_error_word": int(err), "gaussians": view.N}
    view.close()
    tmp = a.out + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(res, fh)
    os.replace(tmp, a.out)
    return 0


if __name__ == "__main__":
    sys.exit(main())
