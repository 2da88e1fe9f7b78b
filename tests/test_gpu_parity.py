"""GPU parity of the rasterizer against the FP64 oracle, through the C ABI.

Projection records (depth key, radius, rectangle, tiles touched), the sorted keys and
values and the tile ranges must match bit for bit; images must match within max-abs
1e-4 (pixels next to a threshold may take either side of it); every gradient tensor
within relative L2 1e-3. Scenes are the seeded workloads of ``scenes`` at full size
(the forward workload and the mapping-step workload) and shrunk variants with ragged
image sizes and several views.
"""
import functools

import numpy as np
import pytest

import oracle
from scenes import make_scene, random_image
from scenes.generate import camera_array
from tests.gpu_common import GRAD_RTOL, check_images, gpu_render, read_discrete, rel_l2, to_np, torch_mods

pytestmark = pytest.mark.gpu

SCENES = {
    "fwd10k": lambda: make_scene("fwd10k"),
    "map100k": lambda: make_scene("map100k"),
    "ragged_tiny": lambda: make_scene("map100k", n=600, W=50, H=37, f=40.0),
    "window_k3": lambda: make_scene("window500k", n=20000, K=3, W=160, H=120, f=130.0),
}
# scenes of the fused-form test only: 3 views of 640x480 are 3600 tiles, more than one wave of the
# compositing kernel's variant without the blocks-per-SM register budget, so the 4-pixel fused
# launch takes the variant compiled for more resident blocks (the scenes above take the other one)
FUSED_ONLY = {
    "window_k3_vga": lambda: make_scene("window500k", n=60000, K=3, W=640, H=480, f=525.0),
}


@functools.lru_cache(maxsize=None)
def scene(name):
    return (SCENES.get(name) or FUSED_ONLY[name])()


@functools.lru_cache(maxsize=None)
def oracle_fwd(name):
    s = scene(name)
    return oracle.forward(s.params(), s.cams, s.W, s.H)


@functools.lru_cache(maxsize=None)
def gpu_fwd(name):
    s = scene(name)
    r, g, ct, out = gpu_render(s.params(), s.cams, s.W, s.H)
    return r, g, ct, out, read_discrete(r)


@pytest.mark.parametrize("name", list(SCENES))
def test_projection_discrete_bit_exact(name):
    m = oracle_fwd(name)["lists"].mirror
    d = gpu_fwd(name)[4]
    # the live items (those that emit pairs) are the oracle's; their records are bit-exact (the
    # others have no records: nothing downstream reads them)
    valid = m.count > 0
    np.testing.assert_array_equal(d["live"], valid)
    np.testing.assert_array_equal(d["count"], m.count)
    np.testing.assert_array_equal(d["radius"][valid], m.radius[valid])
    np.testing.assert_array_equal(d["rect"][valid], m.rect[valid])
    np.testing.assert_array_equal(d["depth_bits"][valid], m.depth_bits[valid])


@pytest.mark.parametrize("name", list(SCENES))
def test_projection_continuous(name):
    s = scene(name)
    ref = oracle.project64(s.params(), s.cams, s.W, s.H)
    d = gpu_fwd(name)[4]
    valid = d["count"] > 0  # the records of items that emit nothing are never written or read
    uv, cn, ref = d["uv"][valid].astype(np.float64), d["conic"][valid].astype(np.float64), ref[valid]
    u = uv[:, 0] + uv[:, 1]
    v = uv[:, 2] + uv[:, 3]
    # compensated (hi + lo) 2D mean: far below the 3e-5 px of a plain binary32 value at 640 px
    assert np.abs(u - ref[:, 0]).max() < 1e-6
    assert np.abs(v - ref[:, 1]).max() < 1e-6
    scale = np.maximum(np.abs(ref[:, 2]), np.abs(ref[:, 4]))
    err = np.abs(cn[:, :3] - ref[:, 2:5]).max(axis=1) / scale
    assert err.max() < 2e-5
    assert (np.abs(cn[:, 3] - ref[:, 5]) / ref[:, 5]).max() < 1e-6


@pytest.mark.parametrize("name", list(SCENES))
def test_sort_and_ranges_bit_exact(name):
    L = oracle_fwd(name)["lists"]
    d = gpu_fwd(name)[4]
    assert d["status"] == 0 and d["err"] == 0
    assert d["total_pairs"] == len(L.keys)
    np.testing.assert_array_equal(d["keys"], L.keys)
    np.testing.assert_array_equal(d["vals"], L.vals)
    np.testing.assert_array_equal(d["ranges"], L.ranges)


@pytest.mark.parametrize("name", list(SCENES))
def test_pair_slots_follow_emission_order(name):
    """Each sorted pair's value is its emission index: a permutation of [0, P) that puts an
    item's pairs in its own block [offset, offset + count), in increasing tile order."""
    d = gpu_fwd(name)[4]
    P = len(d["slots"])
    slots = d["slots"].astype(np.int64)
    assert np.array_equal(np.sort(slots), np.arange(P))
    off = d["offset"].astype(np.int64)[d["item"]]
    cnt = d["count"].astype(np.int64)[d["item"]]
    assert np.all((slots >= off) & (slots < off + cnt))
    tile = (d["keys"] >> np.uint64(32)).astype(np.int64)
    order = np.lexsort((tile, d["item"]))
    s_item, s_slot = d["item"][order], slots[order]
    same = s_item[1:] == s_item[:-1]
    assert np.all(s_slot[1:][same] == s_slot[:-1][same] + 1)


@pytest.mark.parametrize("name", list(SCENES))
def test_forward_images(name):
    orc = oracle_fwd(name)
    out = to_np(gpu_fwd(name)[3])
    rep = check_images(out, orc)
    d = gpu_fwd(name)[4]
    assert abs(d["evals"] - orc["total_evals"]) <= 1e-3 * orc["total_evals"]
    print(name, rep)


def _upstream(name, s):
    K, H, W = s.K, s.H, s.W
    return (random_image(11, (K, 3, H, W)), random_image(12, (K, H, W)), random_image(13, (K, H, W)))


@functools.lru_cache(maxsize=None)
def gpu_bwd(name):
    torch, api = torch_mods()
    s = scene(name)
    r, g, ct, out, _ = gpu_fwd(name)
    gr, gd, gt = (torch.as_tensor(a).cuda() for a in _upstream(name, s))
    grads = r.backward(g, ct, out, gr, gd, gt)
    sg = r.screen_grads()
    torch.cuda.synchronize()
    return to_np(grads), to_np(sg)


@functools.lru_cache(maxsize=None)
def oracle_bwd(name):
    s = scene(name)
    gr, gd, gt = _upstream(name, s)
    return oracle.backward(s.params(), s.cams, s.W, s.H, oracle_fwd(name)["lists"], gr, gd, gt)


@pytest.mark.parametrize("name", list(SCENES))
def test_backward_screen_space(name):
    _, sg = gpu_bwd(name)
    o = oracle_bwd(name)["screen"]
    for gk, ok in (("d_mean2d", "d_uv"), ("d_conic", "d_conic"), ("d_depth", "d_z"), ("d_opacity", "d_opac"),
                   ("d_rgb", "d_rgb")):
        e = rel_l2(sg[gk], o[ok])
        assert e < GRAD_RTOL, (gk, e)


@pytest.mark.parametrize("name", list(SCENES))
def test_backward_parameters_and_pose(name):
    g, _ = gpu_bwd(name)
    o = oracle_bwd(name)
    for k in ("means", "log_scales", "quats", "opacity_logits", "rgb", "pose"):
        e = rel_l2(g[k], o[k])
        assert e < GRAD_RTOL, (k, e)


def test_backward_is_deterministic():
    torch, _ = torch_mods()
    s = scene("map100k")
    r, g, ct, out, _ = gpu_fwd("map100k")
    gr, gd, gt = (torch.as_tensor(a).cuda() for a in _upstream("map100k", s))
    a = r.backward(g, ct, out, gr, gd, gt)
    b = r.backward(g, ct, out, gr, gd, gt)
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_loss_l1_against_oracle():
    torch, api = torch_mods()
    K, H, W = 2, 37, 50
    rgb, rgb_t = random_image(21, (K, 3, H, W), 0, 1), random_image(22, (K, 3, H, W), 0, 1)
    dep, dep_t = random_image(23, (K, H, W), 0, 8), random_image(24, (K, H, W), 0, 8)
    rgb_t[0, 0, :3, :3] = rgb[0, 0, :3, :3]  # equal values: sign(0) = 0
    L, gr, gd = oracle.loss_l1(rgb, dep, rgb_t, dep_t, 0.1)
    r = api.Rasterizer(W, H, K, 1)
    out = {"rgb": torch.as_tensor(rgb).cuda(), "depth": torch.as_tensor(dep).cuda()}
    loss, g_rgb, g_depth = r.loss_l1(out, torch.as_tensor(rgb_t).cuda(), torch.as_tensor(dep_t).cuda())
    assert abs(loss.item() - L) <= 1e-5 * abs(L)
    np.testing.assert_allclose(g_rgb.cpu().numpy(), gr, rtol=1e-6, atol=0)
    np.testing.assert_allclose(g_depth.cpu().numpy(), gd, rtol=1e-6, atol=0)


def test_mapping_step_end_to_end():
    """Loss-driven mapping step at the full map100k size: render, L1 against the
    perturbed-scene target, backward to every parameter."""
    torch, api = torch_mods()
    s = scene("map100k")
    t = s.target
    o_t = oracle.forward(t.params(), t.cams, t.W, t.H)
    o = oracle_fwd("map100k")
    L, gr, gd = oracle.loss_l1(o["rgb"], o["depth"], o_t["rgb"], o_t["depth"], 0.1)
    og = oracle.backward(s.params(), s.cams, s.W, s.H, o["lists"], gr, gd)
    _, _, _, out_t = gpu_render(t.params(), t.cams, t.W, t.H)
    r, g, ct, out, _ = gpu_fwd("map100k")
    loss, g_rgb, g_depth = r.loss_l1(out, out_t["rgb"], out_t["depth"])
    grads = to_np(r.backward(g, ct, out, g_rgb, g_depth))
    assert abs(loss.item() - L) <= 1e-4 * L
    for k in ("means", "log_scales", "quats", "opacity_logits", "rgb", "pose"):
        e = rel_l2(grads[k], og[k])
        assert e < GRAD_RTOL, (k, e)


# ----------------------------------------------------------------------------- edge cases

def test_empty_scene():
    torch, api = torch_mods()
    W, H = 48, 32
    params = (np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), np.zeros((0, 4), np.float32),
              np.zeros(0, np.float32), np.zeros((0, 3), np.float32))
    cam = camera_array(50, 50, 24, 16, np.eye(3), np.zeros(3))
    r, g, ct, out = gpu_render(params, cam, W, H, cap=1024)
    o = to_np(out)
    assert np.all(o["rgb"] == 0) and np.all(o["depth"] == 0) and np.all(o["T"] == 1) and np.all(o["last"] == 0)
    assert r.status()[2] == 0


def test_all_culled_behind_camera():
    s = make_scene("fwd10k", n=300)
    means = s.means.copy()
    means[:, 2] = -means[:, 2]
    params = (means,) + s.params()[1:]
    r, g, ct, out = gpu_render(params, s.cams, s.W, s.H, cap=4096)
    d = read_discrete(r)
    assert d["total_pairs"] == 0 and np.all(d["count"] == 0)
    assert np.all(to_np(out)["T"] == 1)


def test_single_gaussian_covering_every_tile():
    W, H = 100, 70
    params = (np.array([[0.0, 0.0, 2.0]], np.float32), np.array([[0.5, 0.4, 0.3]], np.float32),
              np.array([[0.9, 0.1, -0.2, 0.3]], np.float32), np.array([1.0], np.float32),
              np.array([[0.3, 0.6, 0.9]], np.float32))
    cam = camera_array(60, 60, 50, 35, np.eye(3), np.zeros(3))
    orc = oracle.forward(params, cam, W, H)
    assert orc["lists"].mirror.count[0] == 7 * 5
    r, g, ct, out = gpu_render(params, cam, W, H, cap=1024)
    check_images(to_np(out), orc)
    d = read_discrete(r)
    np.testing.assert_array_equal(d["keys"], orc["lists"].keys)


def test_capacity_overflow_is_reported_and_replanned():
    torch, api = torch_mods()
    s = scene("fwd10k")
    g = api.Gaussians.from_numpy(s.params())
    ct = torch.as_tensor(s.cams).cuda()
    r = api.Rasterizer(s.W, s.H, 1, s.N, pair_capacity=1000)
    out = r.render(g, ct)
    code, err, total, _ = r.status()
    assert code == 3 and err & 1  # GS_ERR_CAPACITY_OVERFLOW
    assert total == len(oracle_fwd("fwd10k")["lists"].keys)
    r.plan(g, ct)
    assert r.cap >= total
    out = r.render(g, ct)
    assert r.status()[0] == 0
    check_images(to_np(out), oracle_fwd("fwd10k"))


def test_nonfinite_input_flagged():
    s = make_scene("fwd10k", n=500)
    means = s.means.copy()
    means[7, 0] = np.nan
    params = (means,) + s.params()[1:]
    r, g, ct, out = gpu_render(params, s.cams, s.W, s.H, cap=1 << 16)
    code, err, _, _ = r.status()
    assert code == 6 and err & 4  # GS_ERR_NONFINITE
    orc = oracle.forward(params, s.cams, s.W, s.H)
    assert orc["lists"].mirror.count[7] == 0
    check_images(to_np(out), orc)


def test_bf16_and_f16_storage_match_dequantised_oracle():
    torch, _ = torch_mods()
    s = make_scene("map100k", n=5000, W=160, H=120, f=130.0)
    for dt in (torch.bfloat16, torch.float16):
        stored = [torch.as_tensor(a).to(dt).float().numpy() for a in s.params()[1:]]
        params = (s.means,) + tuple(stored)  # the exactly dequantised values the oracle consumes
        orc = oracle.forward(params, s.cams, s.W, s.H)
        r, g, ct, out = gpu_render(s.params(), s.cams, s.W, s.H, dtype=dt)
        d = read_discrete(r)
        np.testing.assert_array_equal(d["keys"], orc["lists"].keys)
        check_images(to_np(out), orc)


@pytest.mark.parametrize("name", ["ragged_tiny", "map100k"])
def test_pixels_per_thread_variants_agree(name):
    """Every (forward, backward) pixels-per-thread and chunk-depth variant takes the same decisions: the
    forward outputs are bit-identical; the gradients differ only by the order in which
    pixels are summed in FP32 (relative L2 below 1e-5; the pose gradient, a sum over every
    pair with cancellation, is the most sensitive)."""
    torch, api = torch_mods()
    s = scene(name)
    r, g, ct, _, _ = gpu_fwd(name)
    gr, gd, gt = (torch.as_tensor(a).cuda() for a in _upstream(name, s))
    ref = None
    combos = [(f, b, 0, 0) for f in (1, 2, 4) for b in (1, 2, 4)]
    combos += [(2, 4, 64, 32), (4, 2, 256, 128), (1, 1, 256, 128), (2, 2, 64, 128)]  # chunk depths
    for fpx, bpx, fch, bch in combos:
        r.cfg.fwd_px_per_thread, r.cfg.bwd_px_per_thread = fpx, bpx
        r.cfg.fwd_chunk, r.cfg.bwd_chunk = fch, bch
        out = r.render(g, ct)
        grads = r.backward(g, ct, out, gr, gd, gt)
        got = {**{k: v.clone() for k, v in out.items()}, **{"g_" + k: v for k, v in grads.items()}}
        if ref is None:
            ref = got
        else:
            for k in ref:
                if k.startswith("g_"):
                    e = rel_l2(got[k].cpu().numpy(), ref[k].cpu().numpy())
                    assert e < 1e-5, (fpx, bpx, k, e)
                else:
                    assert torch.equal(ref[k], got[k]), (fpx, bpx, k)
    r.cfg.fwd_px_per_thread, r.cfg.bwd_px_per_thread = 0, 0
    r.cfg.fwd_chunk, r.cfg.bwd_chunk = 0, 0


def test_blocks_per_sm_cap_changes_nothing():
    """A cap on the compositing kernels' resident blocks per SM (padding of their dynamic shared
    memory) changes occupancy only: images and gradients are bit-identical, for the two-launch
    and the one-launch forms."""
    torch, api = torch_mods()
    s = scene("map100k")
    r, g, ct, _, _ = gpu_fwd("map100k")
    gr, gd, gt = (torch.as_tensor(a).cuda() for a in _upstream("map100k", s))
    rgb_t = torch.as_tensor(random_image(23, (s.K, 3, s.H, s.W), 0.0, 1.0)).cuda()
    depth_t = torch.as_tensor(random_image(24, (s.K, s.H, s.W), 0.0, 8.0)).cuda()

    def run():
        out = r.render(g, ct)
        grads = r.backward(g, ct, out, gr, gd, gt)
        o = r.new_outputs()
        g_rgb, g_depth, loss = torch.empty_like(o["rgb"]), torch.empty_like(o["depth"]), torch.zeros(1, device="cuda")
        api.gs_raster_fwd_l1_bwd(r.cfg, r.ws, o["rgb"], o["depth"], o["T"], o["last"], rgb_t, depth_t, g_rgb, g_depth,
                                 loss)
        fused = r.screen_grads()
        torch.cuda.synchronize()
        return {**{k: v.clone() for k, v in out.items()}, **{"g_" + k: v for k, v in grads.items()},
                **{"f_" + k: v for k, v in o.items()}, "f_loss": loss, **{"s_" + k: v for k, v in fused.items()}}
    try:
        r.cfg.fwd_px_per_thread = r.cfg.bwd_px_per_thread = 4
        ref = run()
        for cap in (8, 4, 2):
            r.cfg.raster_blocks_per_sm = cap
            got = run()
            assert r.status()[0] == 0
            for k in ref:
                assert torch.equal(ref[k], got[k]), (cap, k)
    finally:
        r.cfg.raster_blocks_per_sm = 0
        r.cfg.fwd_px_per_thread = r.cfg.bwd_px_per_thread = 0


def test_backward_on_deep_lists():
    """Faint Gaussians (opacity 0.005..0.12): no pixel stops, so every tile's list is composited
    to its end, 200 to 1300 splats deep (many staging chunks per tile, transmittance near 0.1 at
    the end); images and gradients against the oracle."""
    torch, api = torch_mods()
    s = make_scene("map100k", n=6000, W=64, H=48, f=50.0)
    params = list(s.params())
    op = np.random.default_rng(5).uniform(0.005, 0.12, s.N).astype(np.float32)
    params[3] = np.log(op / (1 - op)).astype(np.float32)
    params = tuple(params)
    orc = oracle.forward(params, s.cams, s.W, s.H)
    assert orc["last"].max() > 1000
    gr, gd, gt = _upstream("deep", s)
    og = oracle.backward(params, s.cams, s.W, s.H, orc["lists"], gr, gd, gt)
    r, g, ct, out = gpu_render(params, s.cams, s.W, s.H)
    check_images(to_np(out), orc)
    grads = to_np(r.backward(g, ct, out, *(torch.as_tensor(a).cuda() for a in (gr, gd, gt))))
    assert r.status()[0] == 0
    for k in ("means", "log_scales", "quats", "opacity_logits", "rgb", "pose"):
        e = rel_l2(grads[k], og[k])
        assert e < GRAD_RTOL, (k, e)


@pytest.mark.parametrize("name", ["ragged_tiny", "map100k", "window_k3", "window_k3_vga"])
def test_fused_forward_backward_equals_the_two_calls(name):
    """gs_raster_fwd_l1_bwd (each tile's block continues into its backward pass) equals
    gs_raster_fwd_l1 followed by gs_raster_bwd bit for bit: images, T, last, loss gradient images,
    loss and, through gs_project_bwd, every parameter and pose gradient, for every pixels-per-
    thread and forward chunk depth."""
    torch, api = torch_mods()
    s = scene(name)
    r, g, ct, _, _ = gpu_fwd(name)
    rgb_t = torch.as_tensor(random_image(21, (s.K, 3, s.H, s.W))).cuda().abs()
    depth_t = torch.as_tensor(random_image(22, (s.K, s.H, s.W))).cuda().abs() * 5.0

    def grads_of():
        d = "cuda"
        gr = {"means": torch.empty((s.N, 3), device=d), "log_scales": torch.empty((s.N, 3), device=d),
              "quats": torch.empty((s.N, 4), device=d), "opacity_logits": torch.empty(s.N, device=d),
              "rgb": torch.empty((s.N, 3), device=d), "pose": torch.empty((s.K, 6), device=d)}
        api.gs_project_bwd(r.cfg, g, ct, r.ws, gr, overwrite=True)
        return gr

    def run(fused):
        r.project_and_sort(g, ct)  # fresh binning: clears the record bits of the previous run
        o = r.new_outputs()
        g_rgb, g_depth, loss = torch.empty_like(o["rgb"]), torch.empty_like(o["depth"]), torch.empty(1, device="cuda")
        args = (r.cfg, r.ws, o["rgb"], o["depth"], o["T"], o["last"])
        if fused:
            api.gs_raster_fwd_l1_bwd(*args, rgb_t, depth_t, g_rgb, g_depth, loss)
        else:
            api.gs_raster_fwd_l1(*args, rgb_t, depth_t, g_rgb, g_depth, loss)
            api.gs_raster_bwd(*args, g_rgb, g_depth)
        res = {**{k: v.clone() for k, v in o.items()}, "g_rgb": g_rgb, "g_depth": g_depth, "loss": loss}
        res.update({"d_" + k: v for k, v in grads_of().items()})
        return res

    try:
        for px, fch in ((1, 128), (2, 64), (2, 256), (4, 64), (4, 128), (4, 256)):
            r.cfg.fwd_px_per_thread = r.cfg.bwd_px_per_thread = px
            r.cfg.fwd_chunk = fch
            a, b = run(False), run(True)
            torch.cuda.synchronize()
            assert r.status()[0] == 0
            for k in a:
                assert torch.equal(a[k], b[k]), (name, px, fch, k)
            assert torch.count_nonzero(a["d_means"]).item() > 0
    finally:
        r.cfg.fwd_px_per_thread = r.cfg.bwd_px_per_thread = 0
        r.cfg.fwd_chunk = 0


def test_counting_forward_equals_plain_forward():
    """gs_raster_fwd_stats takes the same decisions and writes the same outputs as
    gs_raster_fwd (bit for bit); only it updates the evaluation counters."""
    torch, api = torch_mods()
    s = scene("map100k")
    r, g, ct, ref, d = gpu_fwd("map100k")
    for px in (1, 2, 4):
        r.cfg.fwd_px_per_thread = px
        a, b = r.new_outputs(), r.new_outputs()
        api.gs_raster_fwd(r.cfg, r.ws, a["rgb"], a["depth"], a["T"], a["last"])
        api.gs_raster_fwd_stats(r.cfg, r.ws, b["rgb"], b["depth"], b["T"], b["last"])
        torch.cuda.synchronize()
        for k in a:
            assert torch.equal(a[k], b[k]), (px, k)
            assert torch.equal(a[k], ref[k]), (px, k)
        assert r.status()[3] == d["evals"]
    r.cfg.fwd_px_per_thread = 0


def test_autotuner_picks_a_variant():
    torch, api = torch_mods()
    from paper_2509_06433_gb300 import autotune
    s = scene("fwd10k")
    r, g, ct, _, _ = gpu_fwd("fwd10k")
    res = autotune.tune(r, g, ct, reps=3)
    assert res["choice"][0] in (1, 2, 4) and res["choice"][1] in (1, 2, 4)
    assert (r.cfg.fwd_px_per_thread, r.cfg.bwd_px_per_thread) == res["choice"]
    assert res["chunks"][0] in (64, 128, 256) and res["chunks"][1] in (32, 64, 128)
    if res["fused"]:  # the one-launch form's backward phase stages a fixed chunk; bwd_chunk keeps the
        # standalone backward's best
        assert res["chunks"] == (r.cfg.fwd_chunk, autotune.FUSED_BWD_CHUNK)
    else:
        assert (r.cfg.fwd_chunk, r.cfg.bwd_chunk) == res["chunks"]
    assert r.fused_compositing == res["fused"] and set(k[0] for k in res["fused_ms"]) == {1, 2, 4}
    assert res["two_launch_ms"] > 0 and all(v > 0 for v in res["fused_ms"].values())
    assert res["blocks_per_sm"] in autotune.BLOCKS_PER_SM and r.cfg.raster_blocks_per_sm == res["blocks_per_sm"]
    assert set(res["blocks_per_sm_ms"]) == set(autotune.BLOCKS_PER_SM)
    if res["fused"]:  # one launch: one pixels-per-thread value for both passes
        assert r.cfg.fwd_px_per_thread == r.cfg.bwd_px_per_thread
    check_images(to_np(r.render(g, ct)), oracle_fwd("fwd10k"))
    r.cfg.fwd_px_per_thread, r.cfg.bwd_px_per_thread = 0, 0
    r.cfg.fwd_chunk, r.cfg.bwd_chunk = 0, 0
    r.cfg.raster_blocks_per_sm = 0
    del r.fused_compositing


def test_aerial_two_views_fp16_storage_forward_and_backward():
    """Aerial workload shape (ground + boxes + large translucent Gaussians, 20 deg down-tilt)
    with FP16 attribute storage over two views, against the oracle on the dequantised values."""
    torch, api = torch_mods()
    s = make_scene("aerial2m", n=30_000, K=2, W=320, H=180, f=225.0)
    stored = [torch.as_tensor(a).to(torch.float16).float().numpy() for a in s.params()[1:]]
    params = (s.means,) + tuple(stored)
    orc = oracle.forward(params, s.cams, s.W, s.H)
    r, g, ct, out = gpu_render(s.params(), s.cams, s.W, s.H, dtype=torch.float16)
    d = read_discrete(r)
    np.testing.assert_array_equal(d["keys"], orc["lists"].keys)
    np.testing.assert_array_equal(d["vals"], orc["lists"].vals)
    check_images(to_np(out), orc)
    gr, gd = random_image(31, (s.K, 3, s.H, s.W)), random_image(32, (s.K, s.H, s.W))
    og = oracle.backward(params, s.cams, s.W, s.H, orc["lists"], gr, gd)
    grads = to_np(r.backward(g, ct, out, torch.as_tensor(gr).cuda(), torch.as_tensor(gd).cuda()))
    for k in ("means", "log_scales", "quats", "opacity_logits", "rgb", "pose"):
        e = rel_l2(grads[k], og[k])
        assert e < GRAD_RTOL, (k, e)


@pytest.mark.parametrize("n,K", [(30_000, 1), (65_536, 2), (80_000, 2), (1, 1)])
def test_depth_sort_sizes(n, K):
    """Depth-sort sizes: 30k items, 131072 = 2^17 items (a whole number of 4-key and 8-key
    sort tiles), 160k and a single item; the pair keys, values and ranges equal the oracle's,
    which fixes the depth order of every emitting item."""
    s = make_scene("window500k", n=n, K=K, W=96, H=64, f=80.0) if n > 1 else None
    if s is None:
        params = (np.array([[0.1, -0.1, 2.0]], np.float32), np.array([[-1.0, -1.2, -1.1]], np.float32),
                  np.array([[1.0, 0.0, 0.0, 0.0]], np.float32), np.array([2.0], np.float32),
                  np.array([[0.2, 0.5, 0.7]], np.float32))
        cams = camera_array(60, 60, 48, 32, np.eye(3), np.zeros(3))
        W, H = 96, 64
    else:
        params, cams, W, H = s.params(), s.cams, s.W, s.H
    r, g, ct, out = gpu_render(params, cams, W, H)
    assert r.layout.bin_sort_launches == 5 + 4 + r.layout.sort_passes
    d = read_discrete(r)
    orc = oracle.forward(params, cams, W, H)
    L = orc["lists"]
    assert d["status"] == 0 and d["total_pairs"] == len(L.keys) > 0
    np.testing.assert_array_equal(d["keys"], L.keys)
    np.testing.assert_array_equal(d["vals"], L.vals)
    np.testing.assert_array_equal(d["ranges"], L.ranges)
    check_images(to_np(out), orc)


def test_large_item_and_pair_counts():
    """700k items (15-key sort tiles for the depth sort) and a 2M pair capacity: keys,
    values and ranges equal the oracle's, and the forward images match."""
    torch, api = torch_mods()
    s = make_scene("window500k", n=350_000, K=2, W=96, H=64, f=80.0)
    r, g, ct, out = gpu_render(s.params(), s.cams, s.W, s.H, cap=2_000_000)
    assert r.layout.bin_sort_launches == 5 + 4 + r.layout.sort_passes
    d = read_discrete(r)
    orc = oracle.forward(s.params(), s.cams, s.W, s.H)
    L = orc["lists"]
    assert d["status"] == 0 and d["total_pairs"] == len(L.keys)
    np.testing.assert_array_equal(d["keys"], L.keys)
    np.testing.assert_array_equal(d["vals"], L.vals)
    np.testing.assert_array_equal(d["ranges"], L.ranges)
    check_images(to_np(out), orc)


def test_loss_fused_forward_equals_forward_then_loss():
    """gs_raster_fwd_l1 writes the forward outputs and the loss gradient images bit for bit
    as gs_raster_fwd followed by gs_loss_l1, and the same loss up to summation order."""
    torch, api = torch_mods()
    s = scene("map100k")
    r, g, ct, ref, d = gpu_fwd("map100k")
    rgb_t = torch.as_tensor(random_image(21, (s.K, 3, s.H, s.W))).cuda()
    depth_t = torch.as_tensor(random_image(22, (s.K, s.H, s.W)) * 5).cuda()
    a = r.new_outputs()
    api.gs_raster_fwd(r.cfg, r.ws, a["rgb"], a["depth"], a["T"], a["last"])
    ga, gda, la = torch.empty_like(a["rgb"]), torch.empty_like(a["depth"]), torch.zeros(1, device="cuda")
    api.gs_loss_l1(r.cfg, a["rgb"], a["depth"], rgb_t, depth_t, ga, gda, la, r.ws)
    for px in (1, 2, 4):
        r.cfg.fwd_px_per_thread = px
        b = r.new_outputs()
        gb, gdb, lb = torch.empty_like(b["rgb"]), torch.empty_like(b["depth"]), torch.zeros(1, device="cuda")
        for _ in range(2):  # twice: the block counter resets itself
            api.gs_raster_fwd_l1(r.cfg, r.ws, b["rgb"], b["depth"], b["T"], b["last"], rgb_t, depth_t, gb, gdb, lb)
        torch.cuda.synchronize()
        for k in a:
            assert torch.equal(a[k], b[k]), (px, k)
        assert torch.equal(ga, gb) and torch.equal(gda, gdb), px
        assert abs(la.item() - lb.item()) <= 1e-5 * abs(la.item()), (px, la.item(), lb.item())
    r.cfg.fwd_px_per_thread = 0


def test_overwritten_gradients_equal_zeroed_accumulated_ones():
    torch, api = torch_mods()
    s = scene("window_k3")
    r, g, ct, out, d = gpu_fwd("window_k3")
    gr, gd, gt = (torch.as_tensor(x).cuda() for x in _upstream("window_k3", s))
    api.gs_raster_bwd(r.cfg, r.ws, out["rgb"], out["depth"], out["T"], out["last"], gr, gd, gt)
    shapes = {"means": (s.N, 3), "log_scales": (s.N, 3), "quats": (s.N, 4), "opacity_logits": (s.N,),
              "rgb": (s.N, 3), "pose": (s.K, 6)}
    acc = {k: torch.zeros(v, device="cuda") for k, v in shapes.items()}
    # NaN in the outputs: overwrite must not read them (uninitialised memory may hold NaN)
    ovr = {k: torch.full(v, float("nan"), device="cuda") for k, v in shapes.items()}
    api.gs_project_bwd(r.cfg, g, ct, r.ws, acc)
    api.gs_project_bwd(r.cfg, g, ct, r.ws, ovr, overwrite=True)
    torch.cuda.synchronize()
    for k in shapes:
        assert torch.equal(acc[k], ovr[k]), k


@pytest.mark.parametrize("with_rgb", [True, False])
def test_occluded_render_matches_the_oracle(with_rgb):
    """gs_raster_fwd_occluded against the oracle's occluded render (external surface at random
    depths inside the scene's depth range): images within the parity tolerance, and a surface
    behind everything gives the plain render bit for bit."""
    torch, api = torch_mods()
    s = scene("window_k3")
    r, g, ct, plain, d = gpu_fwd("window_k3")
    rng = np.random.default_rng(17)
    ext_depth = rng.uniform(1.0, 6.0, (s.K, s.H, s.W)).astype(np.float32)
    ext_rgb = rng.uniform(0, 1, (s.K, 3, s.H, s.W)).astype(np.float32) if with_rgb else None
    out = r.new_outputs()
    api.gs_raster_fwd_occluded(r.cfg, r.ws, out["rgb"], out["depth"], out["T"], out["last"],
                               torch.as_tensor(ext_depth).cuda(),
                               torch.as_tensor(ext_rgb).cuda() if with_rgb else None)
    torch.cuda.synchronize()
    L = oracle_fwd("window_k3")["lists"]
    o = oracle.render_occluded(s.params(), s.cams, s.W, s.H, L.vals, L.ranges, ext_depth, ext_rgb)
    got = to_np(out)
    near = o["near"]
    excluded = near >= 2
    assert excluded.mean() <= 1e-3
    for key in ("rgb", "depth", "T"):
        a = got[key].astype(np.float64)
        p, q = np.abs(a - o[key]), np.abs(a - o["alt_" + key])
        nb = np.broadcast_to(near[:, None], p.shape) if key == "rgb" else near
        ex = np.broadcast_to(excluded[:, None], p.shape) if key == "rgb" else excluded
        tol = 1e-4 * (10.0 if key == "depth" else 1.0)  # depth adds T x ext_depth (up to 6)
        ok = (p <= tol) | ((nb == 1) & (q <= tol)) | ex
        assert ok.all(), (key, int((~ok).sum()))
    assert np.abs(got["rgb"] - to_np(plain)["rgb"]).max() > 0.05  # the surface occludes something
    far = r.new_outputs()
    api.gs_raster_fwd_occluded(r.cfg, r.ws, far["rgb"], far["depth"], far["T"], far["last"],
                               torch.full((s.K, s.H, s.W), float("inf"), device="cuda"), None)
    torch.cuda.synchronize()
    for k in ("rgb", "T", "last"):
        assert torch.equal(far[k], plain[k]), k
