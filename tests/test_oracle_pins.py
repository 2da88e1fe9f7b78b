"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test ties one part of the oracle to a closed form, a brute force, an
invariant of the rendering equation or a finite difference, so that a dropped
term, a wrong sign or index or a transposed operand in the oracle fails here.
The method reading they check: EWA projection of 3D Gaussians (mean,
covariance, opacity; Sec. II-A) and front-to-back alpha compositing of the
tile-sorted lists, differentiated end to end for the mapping optimiser (Fig. 3).
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from scenes import make_scene
from scenes.generate import camera_array, identity_camera

ALPHA_MAX, ALPHA_MIN, T_STOP, DIL = 0.99, 1.0 / 255.0, 1e-4, 0.3


def one_gaussian(mean, log_scales, quat, logit, rgb):
    return (np.array([mean], np.float32), np.array([log_scales], np.float32), np.array([quat], np.float32),
            np.array([logit], np.float32), np.array([rgb], np.float32))


def closed_form_image(u, v, S2, o, rgb, z, W, H, rect, tile=16):
    """Single Gaussian: alpha = min(.99, o exp(-0.5 d^T S2^-1 d)) inside its tile rectangle."""
    inv = np.linalg.inv(S2)
    img = np.zeros((3, H, W))
    dep = np.zeros((H, W))
    T = np.ones((H, W))
    x0, x1, y0, y1 = rect
    for py in range(H):
        for px in range(W):
            if not (x0 <= px // tile < x1 and y0 <= py // tile < y1):
                continue
            d = np.array([u - (px + 0.5), v - (py + 0.5)])
            a = min(ALPHA_MAX, o * math.exp(-0.5 * d @ inv @ d))
            if a < ALPHA_MIN:
                continue
            img[:, py, px] = np.asarray(rgb) * a
            dep[py, px] = z * a
            T[py, px] = 1.0 - a
    return img, dep, T


def rect_of(u, v, r, W, H, tile=16):
    Tx, Ty = -(-W // tile), -(-H // tile)
    xs = [t for t in range(Tx) if tile * t <= u + r and tile * (t + 1) > u - r]
    ys = [t for t in range(Ty) if tile * t <= v + r and tile * (t + 1) > v - r]
    return (xs[0], xs[-1] + 1, ys[0], ys[-1] + 1)


def sigmoid(x):
    return 1.0 / (1.0 + math.exp(-x))


# ----------------------------------------------------------------------------- discrete mirror

def test_expdet_within_one_ulp_of_exp():
    x = np.linspace(-30.0, 10.0, 200001, dtype=np.float32)
    y = oracle.expdet(x).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(y - ref) / ulp) <= 1.0
    assert oracle.expdet(np.array([0.0], np.float32))[0] == 1.0
    assert np.isnan(oracle.expdet(np.array([np.nan], np.float32))[0])


def test_logdet_within_four_ulp_of_log():
    # truncating atanh after s^9 (|s| <= 0.172) errs by < 1e-9 relative; the rest is the
    # rounding of about ten binary32 operations
    x = np.concatenate([np.geomspace(1e-30, 1e30, 200001), np.linspace(0.5, 2.0, 100001)]).astype(np.float32)
    y = oracle.logdet(x).astype(np.float64)
    ref = np.log(x.astype(np.float64))
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    big = np.abs(ref) > 1e-3  # near 1 the error is relative to |ln x| itself
    assert np.max(np.abs(y - ref)[big] / ulp[big]) <= 4.0
    assert np.max(np.abs(y - ref)[~big] / np.abs(ref[~big] + 1e-300)) <= 1e-6
    assert oracle.logdet(np.array([1.0], np.float32))[0] == 0.0
    assert oracle.logdet(np.array([0.0], np.float32))[0] == -np.inf


@pytest.mark.parametrize("z,culled", [(0.1, True), (0.2, True), (0.25, False), (-3.0, True)])
def test_near_plane_cull(z, culled):
    p = one_gaussian((0, 0, z), (-4, -4, -4), (1, 0, 0, 0), 0.0, (1, 1, 1))
    m = oracle.project_mirror(p[0], p[1], p[2], p[3], identity_camera(64, 64, 80.0), 64, 64)
    assert (m.count[0] == 0) == culled


def test_offscreen_cull_and_rect_clamp():
    # far to the right of a 64x64 image: no tile; straddling the edge: rect clamped
    p = one_gaussian((5.0, 0, 2), (-4, -4, -4), (1, 0, 0, 0), 0.0, (1, 1, 1))
    m = oracle.project_mirror(p[0], p[1], p[2], p[3], identity_camera(64, 64, 80.0), 64, 64)
    assert m.count[0] == 0
    p = one_gaussian((0.78, 0, 2), (-1.5, -1.5, -1.5), (1, 0, 0, 0), 0.0, (1, 1, 1))
    m = oracle.project_mirror(p[0], p[1], p[2], p[3], identity_camera(64, 64, 80.0), 64, 64)
    x0, x1, y0, y1 = m.rect[0]
    assert m.count[0] > 0 and x1 == 4 and x0 >= 1


def test_depth_key_is_binary32_depth():
    rng = np.random.default_rng(3)
    means = rng.uniform((-1, -1, 1), (1, 1, 9), size=(500, 3)).astype(np.float32)
    ls = np.full((500, 3), -3.0, np.float32)
    qs = np.tile(np.array([1, 0, 0, 0], np.float32), (500, 1))
    m = oracle.project_mirror(means, ls, qs, np.zeros(500, np.float32), identity_camera(64, 64, 60.0), 64, 64)
    # identity camera: the camera depth is the stored z itself
    assert np.array_equal(m.depth_bits, means[:, 2].view(np.uint32))


def _fp64_sigma2(mean, ls, q, cam, W, H):
    R = cam[4:13].astype(np.float64).reshape(3, 3)
    t = cam[13:16].astype(np.float64)
    fx, fy = float(cam[0]), float(cam[1])
    pc = R @ mean.astype(np.float64) + t
    Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Sig = Rq @ np.diag(np.exp(2.0 * ls.astype(np.float64))) @ Rq.T
    limx, limy = 1.3 * 0.5 * W / fx, 1.3 * 0.5 * H / fy
    tx = np.clip(pc[0] / pc[2], -limx, limx)
    ty = np.clip(pc[1] / pc[2], -limy, limy)
    J = np.array([[fx / pc[2], 0, -fx * tx / pc[2]], [0, fy / pc[2], -fy * ty / pc[2]]])
    return J @ R @ Sig @ R.T @ J.T + DIL * np.eye(2), pc


def test_radius_and_rect_against_fp64_and_brute_force():
    rng = np.random.default_rng(11)
    N, W, H = 400, 96, 80
    means = rng.uniform((-1.5, -1.2, 1.5), (1.5, 1.2, 6), size=(N, 3)).astype(np.float32)
    ls = rng.normal(-3.0, 0.8, size=(N, 3)).astype(np.float32)
    qs = rng.normal(size=(N, 4)).astype(np.float32)
    R, _ = np.linalg.qr(np.eye(3) + 0.1 * rng.normal(size=(3, 3)))
    if np.linalg.det(R) < 0:
        R[:, 0] *= -1
    cam = camera_array(70.0, 72.0, 47.0, 41.0, R, rng.normal(0, 0.1, 3))
    m = oracle.project_mirror(means, ls, qs, np.zeros(N, np.float32), cam, W, H)
    checked = 0
    for g in range(N):
        x0, x1, y0, y1 = m.rect[g]
        if (x1 - x0) * (y1 - y0) == 0:
            continue
        S2, pc = _fp64_sigma2(means[g], ls[g], qs[g] / np.linalg.norm(qs[g].astype(np.float64)), cam, W, H)
        lam = np.linalg.eigvalsh(S2)
        mid = 0.5 * (S2[0, 0] + S2[1, 1])
        disc = 0.25 * (S2[0, 0] - S2[1, 1]) ** 2 + S2[0, 1] ** 2
        lmax = mid + math.sqrt(max(0.1, disc))
        if disc >= 0.1:
            assert abs(lmax - lam[1]) <= 1e-9 * lam[1]
        r64 = 3.0 * math.sqrt(lmax)
        if abs(r64 - round(r64)) > 1e-3:  # away from an integer boundary the ceil must agree
            assert m.radius[g] == math.ceil(r64), g
        u, v = m.uv[g]
        assert abs(u - (cam[0] * pc[0] / pc[2] + cam[2])) < 1e-3
        bu = [float(u) - m.radius[g], float(u) + m.radius[g], float(v) - m.radius[g], float(v) + m.radius[g]]
        if min(abs(b / 16 - round(b / 16)) for b in bu) > 1e-4:
            assert tuple(m.rect[g]) == rect_of(float(u), float(v), int(m.radius[g]), W, H), g
        checked += 1
    assert checked > 100


# ----------------------------------------------------------------------------- closed forms

@pytest.mark.parametrize("case", ["isotropic", "rotated", "off_axis"])
def test_single_gaussian_closed_form(case):
    W, H, f, z = 64, 64, 80.0, 3.0
    cam = identity_camera(W, H, f)
    th = math.radians(30.0)
    if case == "isotropic":
        mean, ls, q = (0.0, 0.0, z), (math.log(0.1),) * 3, (1, 0, 0, 0)
    elif case == "rotated":
        mean, ls, q = (0.0, 0.0, z), (math.log(0.15), math.log(0.05), math.log(0.3)), \
            (math.cos(th / 2), 0, 0, math.sin(th / 2))
    else:
        mean, ls, q = (0.6, -0.4, z), (math.log(0.08),) * 3, (1, 0, 0, 0)
    logit, rgb = 0.5, (0.2, 0.5, 0.9)
    p = one_gaussian(mean, ls, q, logit, rgb)
    p64 = tuple(np.asarray(a, np.float64)[0] for a in p)  # the stored (binary32) values, exactly
    x, y, _ = p64[0]
    s = np.exp(p64[1])
    if case == "isotropic":  # Sigma2 = ((f s / z)^2 + 0.3) I
        S2 = ((f * s[0] / z) ** 2 + DIL) * np.eye(2)
    elif case == "rotated":  # rotation about the optical axis: Sigma2 = (f/z)^2 R2 diag(s0^2, s1^2) R2^T + 0.3 I
        qw, qz = p64[2][0], p64[2][3]
        c2, s2 = (qw * qw - qz * qz) / (qw * qw + qz * qz), 2 * qw * qz / (qw * qw + qz * qz)
        R2 = np.array([[c2, -s2], [s2, c2]])
        S2 = (f / z) ** 2 * R2 @ np.diag([s[0] ** 2, s[1] ** 2]) @ R2.T + DIL * np.eye(2)
    else:  # isotropic off axis: Sigma2 = s^2 J J^T + 0.3 I
        JJt = (f / z) ** 2 * np.array([[1 + x * x / z / z, x * y / z / z], [x * y / z / z, 1 + y * y / z / z]])
        S2 = s[0] ** 2 * JJt + DIL * np.eye(2)
    out = oracle.forward(p, cam, W, H)
    m = out["lists"].mirror
    u, v = f * x / z + W / 2, f * y / z + H / 2
    lmax = np.linalg.eigvalsh(S2)[1]
    r = math.ceil(3 * math.sqrt(lmax))
    assert m.radius[0] == r
    rect = rect_of(u, v, r, W, H)
    assert tuple(m.rect[0]) == rect
    img, dep, T = closed_form_image(u, v, S2, sigmoid(p64[3]), p64[4], z, W, H, rect)
    np.testing.assert_allclose(out["rgb"][0], img, rtol=0, atol=1e-12)
    np.testing.assert_allclose(out["depth"][0], dep, rtol=0, atol=1e-12)
    np.testing.assert_allclose(out["T"][0], T, rtol=0, atol=1e-12)
    assert out["near"].sum() == 0


def test_two_disjoint_gaussians_add():
    W, H, f = 64, 32, 60.0
    cam = identity_camera(W, H, f)
    a = one_gaussian((-0.8, 0.0, 3.0), (-3, -3, -3), (1, 0, 0, 0), 1.0, (1.0, 0.2, 0.1))
    b = one_gaussian((0.8, 0.0, 3.0), (-3, -3.5, -3), (0.9, 0.1, 0.3, 0.2), -0.3, (0.1, 0.3, 1.0))
    both = tuple(np.concatenate([x, y]) for x, y in zip(a, b))
    oa, ob, oab = (oracle.forward(p, cam, W, H) for p in (a, b, both))
    ra, rb = oa["lists"].mirror.rect[0], ob["lists"].mirror.rect[0]
    assert ra[1] <= rb[0]  # disjoint tile rectangles
    np.testing.assert_allclose(oab["rgb"], oa["rgb"] + ob["rgb"], atol=1e-15)
    np.testing.assert_allclose(oab["depth"], oa["depth"] + ob["depth"], atol=1e-15)
    np.testing.assert_allclose(oab["T"], oa["T"] * ob["T"], atol=1e-15)


# ----------------------------------------------------------------------------- brute force

def _brute_render(params, cam, W, H):
    """Per pixel: every Gaussian, ordered by camera depth, composited front to back."""
    means, ls, qs, lg, rgb = (np.asarray(a, np.float64) for a in params)
    R = cam[4:13].astype(np.float64).reshape(3, 3)
    t = cam[13:16].astype(np.float64)
    fx, fy, cx, cy = (float(c) for c in cam[:4])
    recs = []
    for g in range(means.shape[0]):
        S2, pc = _fp64_sigma2(means[g], ls[g], qs[g] / np.linalg.norm(qs[g]), cam, W, H)
        recs.append((pc[2], g, fx * pc[0] / pc[2] + cx, fy * pc[1] / pc[2] + cy, np.linalg.inv(S2),
                     1 / (1 + math.exp(-lg[g])), rgb[g]))
    recs.sort(key=lambda r: (r[0], r[1]))
    img, dep, T = np.zeros((3, H, W)), np.zeros((H, W)), np.ones((H, W))
    for py in range(H):
        for px in range(W):
            Tp, c, d = 1.0, np.zeros(3), 0.0
            for z, g, u, v, inv, o, col in recs:
                dd = np.array([u - px - 0.5, v - py - 0.5])
                pw = -0.5 * dd @ inv @ dd
                if pw > 0:
                    continue
                a = min(ALPHA_MAX, o * math.exp(pw))
                if a < ALPHA_MIN:
                    continue
                if Tp * (1 - a) < T_STOP:
                    break
                c += col * a * Tp
                d += z * a * Tp
                Tp *= 1 - a
            img[:, py, px], dep[py, px], T[py, px] = c, d, Tp
    return img, dep, T


def test_tiled_sorted_render_equals_per_pixel_depth_sort():
    rng = np.random.default_rng(5)
    N, W, H, f = 7, 32, 32, 60.0
    params = (rng.uniform((-0.2, -0.2, 3), (0.2, 0.2, 5), (N, 3)).astype(np.float32),
              rng.normal(-0.3, 0.1, (N, 3)).astype(np.float32),
              rng.normal(size=(N, 4)).astype(np.float32),
              rng.normal(0.5, 1.0, N).astype(np.float32),
              rng.uniform(0, 1, (N, 3)).astype(np.float32))
    cam = identity_camera(W, H, f)
    out = oracle.forward(params, cam, W, H)
    assert np.all(out["lists"].mirror.rect == [0, 2, 0, 2])  # every rect covers the 2x2 tiles
    img, dep, T = _brute_render(params, cam, W, H)
    np.testing.assert_allclose(out["rgb"][0], img, atol=1e-12)
    np.testing.assert_allclose(out["depth"][0], dep, atol=1e-12)
    np.testing.assert_allclose(out["T"][0], T, atol=1e-12)
    assert out["T"].min() < 0.01  # the stop threshold is exercised


def test_binning_against_brute_force_emission_and_lexsort():
    """Given each item's tile set (pinned against FP64 brute force by the two emission-cull
    tests below), the pairs are emitted in (k, g) order, tiles row-major, and stably sorted
    by (tile, depth bits); the ranges delimit each tile's run."""
    from scenes import make_scene
    s = make_scene("map100k", n=3000, W=160, H=120, f=130.0)
    W, H = s.W, s.H
    cams = np.stack([s.cams[0], camera_array(130.0, 130.0, 80, 60,
                                             Rotation.from_euler("y", 8, degrees=True).as_matrix(), (0.1, 0, 0))])
    lists = oracle.discrete(s.params(), cams, W, H)
    m = lists.mirror
    N, K, Tx, Ty = s.N, 2, 10, 8
    tile_all = (lists.keys >> np.uint64(32)).astype(np.int64)
    item_of = (tile_all // (Tx * Ty)) * N + lists.vals.astype(np.int64)
    tiles_of = {}
    for kg, t in zip(item_of, tile_all):
        tiles_of.setdefault(int(kg), []).append(int(t))
    keys, order_idx = [], []
    e = 0
    for kg in range(K * N):
        ts = sorted(tiles_of.get(kg, []))
        assert len(ts) == m.count[kg]
        x0, x1, y0, y1 = m.rect[kg]
        for tid in ts:  # row-major inside the rectangle = increasing tile id
            ty, tx = divmod(tid - (kg // N) * Tx * Ty, Tx)
            assert x0 <= tx < x1 and y0 <= ty < y1
            keys.append((tid << 32) | int(m.depth_bits[kg]))
            order_idx.append((e, kg % N))
            e += 1
    keys = np.array(keys, np.uint64)
    emit = np.array([o[0] for o in order_idx])
    gid = np.array([o[1] for o in order_idx], np.uint32)
    perm = np.lexsort((emit, keys))
    assert np.array_equal(lists.keys, keys[perm])
    assert np.array_equal(lists.vals, gid[perm])
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    cnt = np.bincount(tiles, minlength=K * Tx * Ty)
    r = lists.ranges.astype(np.int64)
    assert np.array_equal(r[:, 1] - r[:, 0], cnt)
    starts = np.concatenate([[0], np.cumsum(cnt)[:-1]])
    nz = cnt > 0
    assert np.array_equal(r[nz, 0], starts[nz])
    assert np.all(r[~nz] == 0)


def _cull_scene(seed, N=400, W=160, H=112, f=140.0):
    """Thin, rotated, large and barely visible Gaussians: many rectangle tiles their
    alpha >= 1/255 ellipse misses."""
    rng = np.random.default_rng(seed)
    means = rng.uniform((-0.9, -0.6, 2.0), (0.9, 0.6, 6.0), (N, 3)).astype(np.float32)
    ls = np.stack([rng.uniform(-4.5, -1.0, N), rng.uniform(-6.0, -2.5, N), rng.uniform(-5.0, -2.0, N)], 1)
    qs = rng.normal(size=(N, 4)).astype(np.float32)
    o = np.where(rng.uniform(size=N) < 0.2, rng.uniform(0.0035, 0.006, N), rng.uniform(0.02, 0.999, N))
    logits = np.log(o / (1 - o)).astype(np.float32)
    rgb = rng.uniform(0, 1, (N, 3)).astype(np.float32)
    return (means, ls.astype(np.float32), qs, logits, rgb), identity_camera(W, H, f), W, H


def _tile_sets(lists, N, Tx, Ty):
    tiles = (lists.keys >> np.uint64(32)).astype(np.int64)
    items = (tiles // (Tx * Ty)) * N + lists.vals.astype(np.int64)
    out = {}
    for kg, t in zip(items, tiles % (Tx * Ty)):
        out.setdefault(int(kg), set()).add(int(t))
    return out


def test_emission_cull_is_conservative():
    """No pixel centre of a rectangle tile left out of an item's emitted tiles reaches
    alpha >= 1/255 (FP64, every pixel of every such tile)."""
    params, cam, W, H = _cull_scene(21)
    lists = oracle.discrete(params, cam, W, H)
    m = lists.mirror
    pr = oracle.project64(params, cam, W, H)
    Tx, Ty = -(-W // 16), -(-H // 16)
    sets = _tile_sets(lists, len(params[0]), Tx, Ty)
    yy, xx = np.mgrid[0:H, 0:W] + 0.5
    culled_tiles = 0
    for g in range(len(params[0])):
        x0, x1, y0, y1 = m.rect[g]
        if (x1 - x0) * (y1 - y0) == 0:
            continue
        u, v, A, B, C, z, o, det = pr[g]
        dx, dy = u - xx, v - yy
        alpha = o * np.exp(-0.5 * (A * dx * dx + 2 * B * dx * dy + C * dy * dy))
        keep = alpha >= 1 / 255
        have = sets.get(g, set())
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                if ty * Tx + tx in have:
                    continue
                culled_tiles += 1
                assert not keep[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16].any(), (g, tx, ty)
    rect_tiles = int(sum((r[1] - r[0]) * (r[3] - r[2]) for r in m.rect))
    assert culled_tiles > 0.25 * rect_tiles  # the cull is exercised


def _min_quadratic_on_box(u, v, P, xlo, xhi, ylo, yhi):
    """min over the box of (p - m)^T P (p - m) for positive definite P (exact, FP64)."""
    if xlo <= u <= xhi and ylo <= v <= yhi:
        return 0.0
    a, b, c = P[0, 0], P[0, 1], P[1, 1]
    best = math.inf
    for y in (ylo, yhi):  # horizontal edges: minimise over x
        dy = y - v
        x = min(max(u - b * dy / a, xlo), xhi)
        dx = x - u
        best = min(best, a * dx * dx + 2 * b * dx * dy + c * dy * dy)
    for x in (xlo, xhi):
        dx = x - u
        y = min(max(v - b * dx / c, ylo), yhi)
        dy = y - v
        best = min(best, a * dx * dx + 2 * b * dx * dy + c * dy * dy)
    return best


def test_emission_cull_is_tight():
    """Every emitted tile's square of pixel centres, widened by the margin, meets the
    ellipse d^T Sigma2^-1 d <= 2 ln(255 o) enlarged by its margin (FP64, exact minimum)."""
    params, cam, W, H = _cull_scene(22)
    lists = oracle.discrete(params, cam, W, H)
    m = lists.mirror
    pr = oracle.project64(params, cam, W, H)
    Tx, Ty = -(-W // 16), -(-H // 16)
    sets = _tile_sets(lists, len(params[0]), Tx, Ty)
    n = 0
    for g, tiles in sets.items():
        u, v, A, B, C, z, o, det = pr[g]
        P = np.array([[A, B], [B, C]])
        L = math.log(255 * o)
        kap = 2 * (L + 0.02 * abs(L) + 1.5e-4)
        S2 = np.linalg.inv(P)
        hx, hy = math.sqrt(kap * S2[0, 0]), math.sqrt(kap * S2[1, 1])
        mx, my = 0.05 + 0.002 * hx + 1e-3, 0.05 + 0.002 * hy + 1e-3
        for t in tiles:
            ty, tx = divmod(t, Tx)
            q = _min_quadratic_on_box(u, v, P, 16 * tx + 0.5 - mx, 16 * tx + 15.5 + mx, 16 * ty + 0.5 - my,
                                      16 * ty + 15.5 + my)
            assert q <= kap * (1 + 1e-4) + 1e-6, (g, tx, ty, q, kap)
            n += 1
    assert n > 500


def test_tiled_render_with_culled_pairs_equals_per_pixel_depth_sort():
    params, cam, W, H = _cull_scene(23, N=60, W=48, H=48, f=45.0)
    out = oracle.forward(params, cam, W, H)
    m = out["lists"].mirror
    rect_tiles = int(sum((r[1] - r[0]) * (r[3] - r[2]) for r in m.rect))
    assert m.count.sum() < 0.85 * rect_tiles  # pairs were culled
    img, dep, T = _brute_render(params, cam, W, H)
    np.testing.assert_allclose(out["rgb"][0], img, atol=1e-12)
    np.testing.assert_allclose(out["depth"][0], dep, atol=1e-12)
    np.testing.assert_allclose(out["T"][0], T, atol=1e-12)


# ----------------------------------------------------------------------------- invariants

def _scene_small(seed, N=40, W=48, H=40, f=50.0, white=False):
    rng = np.random.default_rng(seed)
    params = [rng.uniform((-1, -0.8, 2), (1, 0.8, 5), (N, 3)).astype(np.float32),
              rng.normal(-2.2, 0.4, (N, 3)).astype(np.float32),
              rng.normal(size=(N, 4)).astype(np.float32),
              rng.normal(1.0, 1.5, N).astype(np.float32),
              rng.uniform(0, 1, (N, 3)).astype(np.float32)]
    if white:
        params[4][:] = 1.0
    return tuple(params), identity_camera(W, H, f), W, H


def test_partition_of_unity():
    params, cam, W, H = _scene_small(1, white=True)
    out = oracle.forward(params, cam, W, H)
    for ch in range(3):
        np.testing.assert_allclose(out["rgb"][0, ch], 1.0 - out["T"][0], atol=1e-12)
    assert out["T"].min() < 0.05


def test_transmittance_product_and_weights():
    params, cam, W, H = _scene_small(2)
    out = oracle.forward(params, cam, W, H)
    L = out["lists"]
    rgb = np.asarray(params[4], np.float64)
    order = np.argsort(out["T"][0].ravel())
    picks = [order[0], order[len(order) // 4], order[len(order) // 2], order[(3 * len(order)) // 4]]
    for py, px in (divmod(int(i), W) for i in picks):
        g, a, T, Tf = oracle.pixel_trace(params, cam, W, H, L.vals, L.ranges, 0, px, py)
        assert len(g) > 0
        np.testing.assert_allclose(T, np.concatenate([[1.0], np.cumprod(1 - a)[:-1]]), rtol=1e-13)
        np.testing.assert_allclose(Tf, np.prod(1 - a), rtol=1e-13)
        np.testing.assert_allclose(out["T"][0, py, px], Tf, rtol=1e-13)
        np.testing.assert_allclose(out["rgb"][0, :, py, px], (rgb[g] * (a * T)[:, None]).sum(0), atol=1e-13)
        assert np.all(a >= ALPHA_MIN) and np.all(a <= ALPHA_MAX)


def test_loss_l1_hand_example():
    rgb = np.array([[[[0.5, 0.2]], [[0.1, 0.1]], [[0.9, 0.0]]]])  # K=1, 3 channels, H=1, W=2
    rgb_t = np.array([[[[0.25, 0.2]], [[0.3, 0.1]], [[0.4, 0.5]]]])
    dep, dep_t = np.array([[[2.0, 1.0]]]), np.array([[[1.5, 3.0]]])
    L, gr, gd = oracle.loss_l1(rgb, dep, rgb_t, dep_t, 0.1)
    # |diffs| rgb: 0.25, 0, 0.2, 0, 0.5, 0.5 -> mean over 6 = 1.45/6 ; depth: 0.5, 2 -> 0.1 * 2.5/2
    assert abs(L - (1.45 / 6 + 0.1 * 1.25)) < 1e-15
    np.testing.assert_array_equal(np.sign(gr).ravel(), [1, 0, -1, 0, 1, -1])
    np.testing.assert_allclose(np.abs(gr[gr != 0]), 1 / 6)
    np.testing.assert_allclose(gd.ravel(), [0.1 / 2, -0.1 / 2])


# ----------------------------------------------------------------------------- finite differences

def _fd_scene():
    rng = np.random.default_rng(21)
    N, W, H, f = 12, 40, 32, 40.0
    means = rng.uniform((-0.5, -0.4, 2.0), (0.5, 0.4, 4.0), (N, 3))
    means[0] = (2.6, 0.1, 3.0)      # x/z beyond the Jacobian clamp (0.65), rect still on screen
    means[1] = (0.05, -0.05, 2.5)   # opaque one that reaches the 0.99 clamp
    ls = rng.normal(-2.0, 0.3, (N, 3))
    ls[0] = (-0.3, -0.4, -0.5)
    ls[1] = (-1.8, -1.9, -2.0)
    qs = rng.normal(size=(N, 4)) * rng.uniform(0.5, 2.0, (N, 1))  # not unit length
    lg = rng.normal(0.0, 1.0, N)
    lg[1] = 6.0
    rgb = rng.uniform(0, 1, (N, 3))
    params = tuple(np.asarray(a, np.float32) for a in (means, ls, qs, lg, rgb))
    R = Rotation.from_rotvec([0.05, -0.08, 0.03]).as_matrix()
    cam = camera_array(f, f * 1.05, 21.0, 15.5, R, (0.03, -0.02, 0.1))
    return params, cam, W, H


def _linear_loss(o, w):
    return float((o["rgb"] * w["rgb"]).sum() + (o["depth"] * w["depth"]).sum() + (o["T"] * w["T"]).sum())


def _skew(v):
    return np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])


def test_finite_differences_of_every_parameter_and_the_pose():
    params, cam, W, H = _fd_scene()
    lists = oracle.discrete(params, cam, W, H)
    p64 = [np.asarray(a, np.float64).copy() for a in params]
    base = oracle.render_fwd(p64, cam, W, H, lists.vals, lists.ranges)
    rng = np.random.default_rng(7)
    w = {"rgb": rng.normal(size=base["rgb"].shape), "depth": rng.normal(size=base["depth"].shape),
         "T": rng.normal(size=base["T"].shape)}
    g = oracle.backward(p64, cam, W, H, lists, w["rgb"], w["depth"], w["T"])
    # the clamp cases of the scene are live
    assert np.abs(g["means"][0]).sum() > 0 and np.abs(g["means"][1]).sum() > 0
    h = 1e-6

    def L_at(pp, c=cam):
        o = oracle.render_fwd(pp, c, W, H, lists.vals, lists.ranges)
        same = np.array_equal(o["evals"], base["evals"]) and np.array_equal(o["last"], base["last"])
        return _linear_loss(o, w), same

    names = ["means", "log_scales", "quats", "opacity_logits", "rgb"]
    n_checked = 0
    for bi, name in enumerate(names):
        an = g[name].reshape(-1)
        scale = np.abs(an).max()
        for j in range(an.size):
            pp = [a.copy() for a in p64]
            flat = pp[bi].reshape(-1)
            flat[j] += h
            Lp, okp = L_at(pp)
            flat[j] -= 2 * h
            Lm, okm = L_at(pp)
            if not (okp and okm):
                continue
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - an[j]) <= 2e-6 * scale + 1e-5 * abs(an[j]), (name, j, fd, an[j])
            n_checked += 1
    assert n_checked >= 0.95 * sum(a.size for a in params)
    # pose: left perturbation T <- (I + xi^) T, translation first
    R = cam[4:13].astype(np.float64).reshape(3, 3)
    t = cam[13:16].astype(np.float64)
    an = g["pose"][0]
    for j in range(6):
        xi = np.zeros(6)
        xi[j] = h
        vals = []
        for sgn in (1, -1):
            E = np.eye(3) + sgn * _skew(xi[3:])
            c = cam.astype(np.float64).copy()
            c[4:13] = (E @ R).reshape(9)
            c[13:16] = E @ t + sgn * xi[:3]
            vals.append(L_at(p64, c)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - an[j]) <= 2e-6 * np.abs(an).max() + 1e-5 * abs(an[j]), (j, fd, an[j])


def test_pose_translation_gradient_equals_summed_mean_gradient():
    params, cam, W, H = _fd_scene()
    lists = oracle.discrete(params, cam, W, H)
    rng = np.random.default_rng(8)
    gr = rng.normal(size=(1, 3, H, W))
    gd = rng.normal(size=(1, H, W))
    g = oracle.backward(params, cam, W, H, lists, gr, gd)
    R = cam[4:13].astype(np.float64).reshape(3, 3)
    # moving every mean by delta in the world moves p_c by R delta, exactly like rho = R delta
    np.testing.assert_allclose(g["means"].sum(0), R.T @ g["pose"][0, :3], rtol=1e-10, atol=1e-12)


def test_two_views_sum_single_view_gradients():
    params, cam, W, H = _fd_scene()
    cam2 = camera_array(42.0, 42.0, 20.0, 16.0, Rotation.from_rotvec([0, 0.1, 0]).as_matrix(), (0.1, 0, 0.2))
    cams = np.stack([cam, cam2])
    rng = np.random.default_rng(9)
    gr = rng.normal(size=(2, 3, H, W))
    gd = rng.normal(size=(2, H, W))
    both = oracle.backward(params, cams, W, H, oracle.discrete(params, cams, W, H), gr, gd)
    singles = [oracle.backward(params, c, W, H, oracle.discrete(params, c, W, H), gr[k:k + 1], gd[k:k + 1])
               for k, c in enumerate(cams)]
    for name in ("means", "log_scales", "quats", "opacity_logits", "rgb"):
        np.testing.assert_allclose(both[name], singles[0][name] + singles[1][name], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(both["pose"], np.concatenate([s["pose"] for s in singles]), rtol=1e-10, atol=1e-12)


# ----------------------------------------------------------------------------- occlusion

def _brute_occluded(params, cam, W, H, ext_depth, ext_rgb):
    """Per pixel: every Gaussian in front of the external surface, by depth, front to back; then
    the surface through the remaining transmittance."""
    means, ls, qs, lg, rgb = (np.asarray(a, np.float64) for a in params)
    fx, fy, cx, cy = (float(c) for c in cam[:4])
    recs = []
    for g in range(means.shape[0]):
        S2, pc = _fp64_sigma2(means[g], ls[g], qs[g] / np.linalg.norm(qs[g]), cam, W, H)
        recs.append((pc[2], g, fx * pc[0] / pc[2] + cx, fy * pc[1] / pc[2] + cy, np.linalg.inv(S2),
                     1 / (1 + math.exp(-lg[g])), rgb[g]))
    recs.sort(key=lambda r: (r[0], r[1]))
    img, dep, T = np.zeros((3, H, W)), np.zeros((H, W)), np.ones((H, W))
    for py in range(H):
        for px in range(W):
            Tp, c, d = 1.0, np.zeros(3), 0.0
            zmax = float(ext_depth[py, px])
            for z, g, u, v, inv, o, col in recs:
                if z >= zmax:
                    break
                dd = np.array([u - px - 0.5, v - py - 0.5])
                pw = -0.5 * dd @ inv @ dd
                if pw > 0:
                    continue
                a = min(ALPHA_MAX, o * math.exp(pw))
                if a < ALPHA_MIN:
                    continue
                if Tp * (1 - a) < T_STOP:
                    break
                c += col * a * Tp
                d += z * a * Tp
                Tp *= 1 - a
            img[:, py, px] = c + Tp * ext_rgb[:, py, px]
            dep[py, px], T[py, px] = d + Tp * zmax, Tp
    return img, dep, T


def test_occluded_render_equals_per_pixel_brute_force():
    rng = np.random.default_rng(9)
    N, W, H, f = 9, 32, 32, 60.0
    params = (rng.uniform((-0.2, -0.2, 3), (0.2, 0.2, 5), (N, 3)).astype(np.float32),
              rng.normal(-0.3, 0.1, (N, 3)).astype(np.float32),
              rng.normal(size=(N, 4)).astype(np.float32),
              rng.normal(0.5, 1.0, N).astype(np.float32),
              rng.uniform(0, 1, (N, 3)).astype(np.float32))
    cam = identity_camera(W, H, f)
    ext_depth = rng.uniform(2.5, 5.5, (1, H, W)).astype(np.float32)
    ext_rgb = rng.uniform(0, 1, (1, 3, H, W)).astype(np.float32)
    lists = oracle.discrete(params, cam, W, H)
    o = oracle.render_occluded(params, cam, W, H, lists.vals, lists.ranges, ext_depth, ext_rgb)
    img, dep, T = _brute_occluded(params, cam, W, H, ext_depth[0], ext_rgb[0].astype(np.float64))
    ok = o["near"][0] == 0
    assert ok.mean() > 0.99
    np.testing.assert_allclose(o["rgb"][0][:, ok], img[:, ok], atol=1e-12)
    np.testing.assert_allclose(o["depth"][0][ok], dep[ok], atol=1e-12)
    np.testing.assert_allclose(o["T"][0][ok], T[ok], atol=1e-12)
    # occluded pixels exist, and pixels whose surface is behind everything equal the plain render
    plain = oracle.render_fwd(params, cam, W, H, lists.vals, lists.ranges)
    far = oracle.render_occluded(params, cam, W, H, lists.vals, lists.ranges, np.full((1, H, W), 1e9, np.float32))
    np.testing.assert_array_equal(far["T"], plain["T"])
    np.testing.assert_array_equal(far["rgb"], plain["rgb"] + plain["T"][:, None] * 0.0)
    assert np.abs(o["rgb"] - plain["rgb"]).max() > 0.05
    near = oracle.render_occluded(params, cam, W, H, lists.vals, lists.ranges, np.full((1, H, W), 0.5, np.float32),
                                  ext_rgb)
    np.testing.assert_array_equal(near["rgb"], ext_rgb.astype(np.float64))
    assert np.all(near["T"] == 1.0) and np.all(near["depth"] == 0.5)


def test_render_tiles_equals_full_render():
    # the tile-sampled FP64 render (full-size parity on sampled outputs) is the full render
    # restricted to those tiles, element for element
    s = make_scene("map100k", n=3000, W=72, H=50, f=60.0)
    o = oracle.forward(s.params(), s.cams, s.W, s.H)
    L = o["lists"]
    Tx, Ty = (s.W + 15) // 16, (s.H + 15) // 16
    tiles = np.array([0, 3, Tx + 2, Tx * Ty - 1])  # includes ragged edge tiles
    t = oracle.render_tiles(s.params(), s.cams, s.W, s.H, L.vals, L.ranges, tiles)
    for i, tg in enumerate(tiles):
        ty, tx = divmod(int(tg), Tx)
        ys, xs = slice(ty * 16, min(ty * 16 + 16, s.H)), slice(tx * 16, min(tx * 16 + 16, s.W))
        h, w = ys.stop - ys.start, xs.stop - xs.start
        assert np.array_equal(t["rgb"][i][:, :h, :w], o["rgb"][0][:, ys, xs])
        for k in ("depth", "T", "last", "near", "alt_T", "alt_depth", "alt_last"):
            assert np.array_equal(t[k][i][:h, :w], o[k][0][ys, xs]), k
        assert np.all(t["near"][i][h:, :] == -1) and np.all(t["near"][i][:, w:] == -1)
