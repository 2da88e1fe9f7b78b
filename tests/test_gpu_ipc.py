"""The map shared over CUDA IPC with a viewer process (Sec. III, Fig. 5): the viewer's frames
of a static shared map equal the exporter's own render bit for bit and, at the paper's stereo
672x376, the FP64 oracle's render of the map at the viewer's poses; the viewer keeps rendering
while the exporter's mapping graph updates the map, and pauses / resumes on request."""
import json
import os
import subprocess
import sys
import time

import numpy as np
import pytest

from scenes import make_scene

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def spawn_viewer(tmp_path, desc, *extra):
    dpath = tmp_path / "map.json"
    dpath.write_text(json.dumps(desc))
    out, ready = tmp_path / "viewer.json", tmp_path / "ready"
    cmd = [sys.executable, "-m", "paper_2509_06433_gb300.viewer", "--desc", str(dpath), "--out", str(out),
           "--ready", str(ready), *extra]
    proc = subprocess.Popen(cmd, cwd=ROOT, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    return proc, out, ready


def finish(proc, timeout=240):
    try:
        log, _ = proc.communicate(timeout=timeout)
    except subprocess.TimeoutExpired:
        proc.kill()  # our own child
        log, _ = proc.communicate()
        pytest.fail("viewer did not finish:\n" + log.decode(errors="replace")[-2000:])
    assert proc.returncode == 0, log.decode(errors="replace")[-2000:]


def test_viewer_frames_equal_exporter_render(tmp_path):
    import torch
    from paper_2509_06433_gb300 import api, ipc
    s = make_scene("map100k", n=20_000, W=160, H=120, f=130.0)
    shared = ipc.SharedMap(s.N)
    shared.load(api.Gaussians.from_numpy(s.params()))
    shared.publish()
    torch.cuda.synchronize()
    from paper_2509_06433_gb300.viewer import orbit_rig
    cams = orbit_rig(7, 2, (0.0, 0.0, 5.0), 4.0, 130.0, 160, 120)
    np.save(tmp_path / "cams.npy", cams)
    proc, out, _ = spawn_viewer(tmp_path, shared.descriptor(), "--cams", str(tmp_path / "cams.npy"), "--frames",
                                "3", "--width", "160", "--height", "120", "--save", str(tmp_path / "frame.npz"))
    finish(proc)
    got = np.load(tmp_path / "frame.npz")["rgb"]
    r = api.Rasterizer(160, 120, 2, s.N)
    ct = torch.as_tensor(cams).cuda()
    r.plan(shared.g, ct)
    mine = r.render(shared.g, ct)["rgb"].cpu().numpy()
    assert got.shape == mine.shape and np.array_equal(got, mine)
    assert mine.max() > 0.1
    res = json.loads(out.read_text())
    assert res["device_error_word"] == 0 and res["frames"] == 3
    shared.close()


def test_viewer_frames_match_the_oracle_at_the_viewer_poses(tmp_path):
    """The viewer process renders the whole shared map100k map (100k Gaussians) as a stereo pair
    at the paper's 672x376 (eyes 64 mm apart); every pixel of both eyes (RGB, depth, T, last
    contributor) is compared with the FP64 oracle's render at those poses."""
    import torch
    from paper_2509_06433_gb300 import api, ipc
    from paper_2509_06433_gb300.viewer import orbit_rig
    from tests.gpu_common import check_images
    import oracle
    s = make_scene("map100k")
    shared = ipc.SharedMap(s.N)
    shared.load(api.Gaussians.from_numpy(s.params()))
    shared.publish()
    torch.cuda.synchronize()
    cams = orbit_rig(31, 2, (0.0, 0.0, 5.0), 4.0, 336.0, 672, 376)
    np.save(tmp_path / "cams.npy", cams)
    proc, out, _ = spawn_viewer(tmp_path, shared.descriptor(), "--cams", str(tmp_path / "cams.npy"), "--frames",
                                "2", "--width", "672", "--height", "376", "--save", str(tmp_path / "frame.npz"))
    finish(proc)
    got = dict(np.load(tmp_path / "frame.npz"))
    res = json.loads(out.read_text())
    assert res["device_error_word"] == 0
    o = oracle.forward(s.params(), cams, 672, 376)
    rep = check_images(got, o)
    assert got["rgb"].shape == (2, 3, 376, 672) and got["rgb"].max() > 0.1
    assert (got["last"] > 0).mean() > 0.5, "the viewpoints must see the map"
    print(f"\nviewer vs oracle, stereo 672x376: rgb {rep['rgb']:.2e} depth {rep['depth']:.2e} T {rep['T']:.2e}")
    shared.close()


def test_viewer_pauses_and_resumes_on_control(tmp_path):
    """With --control the viewer renders only while the control file exists and ends at the stop
    file; the frames it reports are the ones it rendered while active."""
    import torch
    from paper_2509_06433_gb300 import api, ipc
    s = make_scene("map100k", n=20_000, W=160, H=120, f=130.0)
    shared = ipc.SharedMap(s.N)
    shared.load(api.Gaussians.from_numpy(s.params()))
    shared.publish()
    torch.cuda.synchronize()
    control, stop = tmp_path / "render", tmp_path / "stop"
    proc, out, ready = spawn_viewer(tmp_path, shared.descriptor(), "--control", str(control), "--stop", str(stop),
                                    "--width", "160", "--height", "120")
    deadline = time.time() + 240
    while not ready.exists():
        assert proc.poll() is None, proc.communicate()[0].decode(errors="replace")[-2000:]
        assert time.time() < deadline
        time.sleep(0.05)
    time.sleep(0.3)  # paused: no frames
    control.write_text("")
    time.sleep(0.5)  # active
    control.unlink()
    time.sleep(0.3)
    stop.write_text("")
    finish(proc)
    res = json.loads(out.read_text())
    assert res["frames"] > 10 and res["device_error_word"] == 0
    assert 0 < res["seconds"] < 0.75  # the active time only
    shared.close()


def test_viewer_runs_while_the_map_is_optimised(tmp_path):
    import torch
    from paper_2509_06433_gb300 import api, ipc
    from paper_2509_06433_gb300.tracking import MappingStep
    s = make_scene("map100k", n=30_000, W=320, H=240, f=260.0)
    shared = ipc.SharedMap(s.N)
    shared.load(api.Gaussians.from_numpy(s.params()))
    cams = torch.as_tensor(s.cams).cuda()
    t = s.target
    r = api.Rasterizer(s.W, s.H, 1, s.N)
    gt = api.Gaussians.from_numpy(t.params())
    r.plan(gt, cams)
    tgt = r.render(gt, cams)
    rgb_t, depth_t = tgt["rgb"].clone(), tgt["depth"].clone()
    r.plan(shared.g, cams)
    opt = api.MapOptimizer(shared.g)
    step = MappingStep(r, shared.g, cams, rgb_t, depth_t, graph=True, optimizer=opt)
    shared.publish()
    torch.cuda.synchronize()
    proc, out, ready = spawn_viewer(tmp_path, shared.descriptor(), "--frames", "120")
    deadline = time.time() + 240
    while not ready.exists():
        assert proc.poll() is None, proc.communicate()[0].decode(errors="replace")[-2000:]
        assert time.time() < deadline
        time.sleep(0.05)
    losses, iters = [], 0
    while time.time() < deadline:
        for _ in range(20):
            step.replay()
            shared.publish()
        iters += 20
        losses.append(step.loss.item())
        if out.exists() and iters >= 60:
            break
    finish(proc)
    res = json.loads(out.read_text())
    assert res["frames"] == 120 and res["fps"] > 10 and res["device_error_word"] == 0
    assert iters >= 20 and losses[-1] < losses[0]
    shared.close()
