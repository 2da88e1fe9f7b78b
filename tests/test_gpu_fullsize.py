"""Parity at the full sizes of the benchmark's secondary workloads, in the configuration the
benchmark launches (autotuned compositing variants, reduced-precision storage where the
workload stores it): the sorted keys, values and tile ranges of the whole scene bit-exact
against the oracle; images on sampled tiles (every pixel of each) within 1e-4 of the FP64
oracle; gradients through the identity sum_g dL/dmean_g = sum_k R_k^T dL/drho_k, which holds
at any size (a world translation is a translation of every camera)."""
import numpy as np
import pytest

import oracle
from scenes import make_scene, random_image
from tests.gpu_common import check_images, read_discrete, torch_mods

pytestmark = pytest.mark.gpu

CASES = {
    "track300k": ("f32", 6),
    "window500k": ("bf16", 3),
    "aerial2m": ("f16", 2),
}


def setup_case(name):
    torch, api = torch_mods()
    from paper_2509_06433_gb300 import autotune
    storage, tiles_per_view = CASES[name]
    s = make_scene(name)
    cams_np = s.track_cams if name == "track300k" else s.cams
    dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[storage]
    g = api.Gaussians.from_numpy(s.params(), dtype=dt)
    # the oracle consumes the stored (dequantised) attributes
    params = tuple(t.float().cpu().numpy() for t in (g.means, g.log_scales, g.quats, g.opacity_logits, g.rgb))
    cams = torch.as_tensor(np.ascontiguousarray(cams_np.reshape(-1, 16))).cuda()
    r = api.Rasterizer(s.W, s.H, cams.shape[0], s.N)
    r.plan(g, cams, headroom=1.2)
    autotune.tune(r, g, cams)
    out = r.render(g, cams)
    torch.cuda.synchronize()
    return s, params, cams_np.reshape(-1, 16), g, cams, r, out, tiles_per_view


@pytest.mark.parametrize("name", list(CASES))
def test_full_size_lists_images_and_gradient_identity(name):
    torch, api = torch_mods()
    s, params, cams_np, g, cams, r, out, tpv = setup_case(name)
    K, W, H = cams_np.shape[0], s.W, s.H
    d = read_discrete(r)
    assert d["status"] == 0
    L = oracle.discrete(params, cams_np, W, H)
    assert d["total_pairs"] == len(L.keys)
    np.testing.assert_array_equal(d["keys"], L.keys)
    np.testing.assert_array_equal(d["vals"], L.vals)
    np.testing.assert_array_equal(d["ranges"], L.ranges)
    # images on sampled tiles (every pixel), against the FP64 render of those tiles
    Tx, Ty = r.layout.tiles_x, r.layout.tiles_y
    rng = np.random.default_rng(5)
    tiles = np.concatenate([k * Tx * Ty + rng.choice(Tx * Ty, tpv, replace=False) for k in range(K)])
    o = oracle.render_tiles(params, cams_np, W, H, L.vals, L.ranges, tiles)
    gpu = {k: v.cpu().numpy() for k, v in out.items()}
    got = {"rgb": np.empty_like(o["rgb"]), "depth": np.empty_like(o["depth"]), "T": np.empty_like(o["T"]),
           "last": np.empty_like(o["last"])}
    for i, tg in enumerate(tiles):
        k, rem = divmod(int(tg), Tx * Ty)
        ty, tx = divmod(rem, Tx)
        ys, xs = slice(ty * 16, ty * 16 + 16), slice(tx * 16, tx * 16 + 16)
        got["rgb"][i] = gpu["rgb"][k][:, ys, xs]
        got["depth"][i], got["T"][i], got["last"][i] = gpu["depth"][k][ys, xs], gpu["T"][k][ys, xs], gpu["last"][k][ys, xs]
    assert np.all(o["near"] >= 0)  # the sampled tiles lie inside the image (sizes are multiples of 16)
    check_images(got, o)
    # gradients: the translation identity over every Gaussian and view
    gr = torch.as_tensor(random_image(31, (K, 3, H, W))).cuda()
    gd = torch.as_tensor(random_image(32, (K, H, W))).cuda()
    grads = r.backward(g, cams, out, gr, gd)
    sm = grads["means"].double().sum(0).cpu().numpy()
    R = cams_np[:, 4:13].astype(np.float64).reshape(-1, 3, 3)
    rho = grads["pose"][:, :3].double().cpu().numpy()
    rhs = np.einsum("kji,kj->i", R, rho)
    assert np.abs(sm - rhs).max() <= 1e-4 * np.abs(rhs).max() + 1e-6, (sm, rhs)
    assert np.abs(rhs).max() > 0
