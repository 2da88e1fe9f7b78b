"""Seeded synthetic scenes shaped like the paper's indoor / aerial mapping workloads.

The paper evaluates on its own recorded flight-arena RGB-D sequence (672x376,
ZED 2i camera tilted 20 degrees down, Sec. IV and V), which is not available.
These generators stand in for it with the five workload shapes the hot path is
measured on. Every array is drawn from ``numpy.random.default_rng(seed)``.

Layouts (all float32, structure of arrays, C-contiguous):
  means           [N, 3]  world position (m)
  log_scales      [N, 3]  per-axis log standard deviation (m)
  quats           [N, 4]  rotation quaternion (w, x, y, z)
  opacity_logits  [N]     logit of the opacity
  rgb             [N, 3]  colour (spherical-harmonic degree 0: the colour itself)
  cams            [K, 16] fx, fy, cx, cy, R (3x3 row-major, world->camera), t (3)

Camera frame: x right, y down, z forward (pinhole, pixel centres at i + 0.5).
Rotations are composed with scipy's ``Rotation`` (a library primitive);
nothing here projects, composites or differentiates.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.spatial.transform import Rotation


@dataclasses.dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    rgb: np.ndarray
    cams: np.ndarray
    W: int
    H: int
    name: str = ""
    target: "Scene | None" = None  # perturbed copy rendered as the photometric target
    track_cams: "np.ndarray | None" = None  # perturbed start pose for tracking workloads

    @property
    def N(self) -> int:
        return int(self.means.shape[0])

    @property
    def K(self) -> int:
        return int(self.cams.shape[0])

    def params(self):
        return (self.means, self.log_scales, self.quats, self.opacity_logits, self.rgb)

    def subset(self, idx) -> "Scene":
        return dataclasses.replace(
            self,
            means=np.ascontiguousarray(self.means[idx]),
            log_scales=np.ascontiguousarray(self.log_scales[idx]),
            quats=np.ascontiguousarray(self.quats[idx]),
            opacity_logits=np.ascontiguousarray(self.opacity_logits[idx]),
            rgb=np.ascontiguousarray(self.rgb[idx]),
            target=None,
        )


# ----------------------------------------------------------------------------- cameras

def look_at(position, forward):
    """World->camera (R, t) for a camera at ``position`` looking along ``forward``.

    World z is up; the camera's y axis points down the image.
    """
    f = np.asarray(forward, np.float64)
    f = f / np.linalg.norm(f)
    down = np.array([0.0, 0.0, -1.0])
    r = np.cross(down, f)
    if np.linalg.norm(r) < 1e-9:  # looking straight down/up: pick any right axis
        r = np.array([1.0, 0.0, 0.0])
    r = r / np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ np.asarray(position, np.float64)
    return R, t


def camera_array(fx, fy, cx, cy, R, t) -> np.ndarray:
    c = np.zeros(16, np.float64)
    c[0:4] = (fx, fy, cx, cy)
    c[4:13] = np.asarray(R, np.float64).reshape(9)
    c[13:16] = np.asarray(t, np.float64).reshape(3)
    return c.astype(np.float32)


def identity_camera(W, H, f):
    return camera_array(f, f, W / 2.0, H / 2.0, np.eye(3), np.zeros(3))


def perturb_pose(cam: np.ndarray, rng, rot_deg: float, trans_m: float) -> np.ndarray:
    """Left-multiply a world->camera pose by a rotation of ``rot_deg`` about a random
    axis and a translation of ``trans_m`` in a random direction."""
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    dR = Rotation.from_rotvec(axis * math.radians(rot_deg)).as_matrix()
    R = cam[4:13].astype(np.float64).reshape(3, 3)
    t = cam[13:16].astype(np.float64)
    out = cam.copy()
    out[4:13] = (dR @ R).reshape(9).astype(np.float32)
    out[13:16] = (dR @ t + trans_m * d).astype(np.float32)
    return out


# ----------------------------------------------------------------------------- gaussians

def _unit_quats(rng, n):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _free(rng, n, lo, hi, ls_mu=-3.0, ls_sd=0.5, logit_mu=0.0, logit_sd=1.0):
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    return dict(
        means=rng.uniform(lo, hi, size=(n, 3)),
        log_scales=rng.normal(ls_mu, ls_sd, size=(n, 3)),
        quats=_unit_quats(rng, n),
        opacity_logits=rng.normal(logit_mu, logit_sd, size=n),
        rgb=rng.uniform(0.0, 1.0, size=(n, 3)),
    )


def _on_plane(rng, n, center, frame: Rotation, half_a, half_b,
              normal_ls=(-6.0, 0.3), inplane_ls=(-3.0, 0.5), logit=(0.0, 1.0)):
    """Gaussians lying on a plane: the frame's third axis is the plane normal."""
    basis = frame.as_matrix()
    a = rng.uniform(-half_a, half_a, size=n)
    b = rng.uniform(-half_b, half_b, size=n)
    means = np.asarray(center, np.float64)[None, :] + a[:, None] * basis[:, 0] + b[:, None] * basis[:, 1]
    theta = rng.uniform(0.0, 2.0 * math.pi, size=n)
    rots = frame * Rotation.from_rotvec(np.stack([np.zeros(n), np.zeros(n), theta], axis=1))
    xyzw = rots.as_quat()
    quats = np.concatenate([xyzw[:, 3:4], xyzw[:, 0:3]], axis=1)
    ls = np.empty((n, 3))
    ls[:, 0:2] = rng.normal(inplane_ls[0], inplane_ls[1], size=(n, 2))
    ls[:, 2] = rng.normal(normal_ls[0], normal_ls[1], size=n)
    return dict(means=means, log_scales=ls, quats=quats,
                opacity_logits=rng.normal(logit[0], logit[1], size=n),
                rgb=rng.uniform(0.0, 1.0, size=(n, 3)))


def _concat(parts):
    keys = parts[0].keys()
    return {k: np.concatenate([p[k] for p in parts], axis=0) for k in keys}


def _to_scene(d, cams, W, H, name) -> Scene:
    f32 = lambda a: np.ascontiguousarray(np.asarray(a, np.float32))  # noqa: E731
    return Scene(f32(d["means"]), f32(d["log_scales"]), f32(d["quats"]),
                 f32(d["opacity_logits"]), f32(d["rgb"]),
                 f32(np.stack(cams) if isinstance(cams, list) else cams), W, H, name)


def _perturbed_copy(rng, s: Scene, mean_sd=0.01, rgb_sd=0.05) -> Scene:
    return dataclasses.replace(
        s,
        means=(s.means + rng.normal(0.0, mean_sd, size=s.means.shape)).astype(np.float32),
        rgb=(s.rgb + rng.normal(0.0, rgb_sd, size=s.rgb.shape)).astype(np.float32),
        target=None,
    )


def _plane_mixture(rng, n, n_planes=3):
    """Half free Gaussians in the box, half on random planes crossing the frustum."""
    n_free = n // 2
    parts = [_free(rng, n_free, (-2, -2, 2), (2, 2, 8))]
    rest = n - n_free
    per = [rest // n_planes + (1 if i < rest % n_planes else 0) for i in range(n_planes)]
    for m in per:
        center = rng.uniform((-1.0, -1.0, 3.5), (1.0, 1.0, 6.5))
        parts.append(_on_plane(rng, m, center, Rotation.random(random_state=rng), 2.5, 2.5))
    return _concat(parts)


def _room(rng, n):
    """Six walls of an 8 x 6 x 3 m room (x in [0,8], y in [0,6], z in [0,3]) + 10% free."""
    n_free = n // 10
    rest = n - n_free
    L, Wd, Hh = 8.0, 6.0, 3.0
    faces = [  # (center, frame whose third axis is the normal, half extents)
        ((L / 2, Wd / 2, 0.0), Rotation.identity(), L / 2, Wd / 2),
        ((L / 2, Wd / 2, Hh), Rotation.from_euler("x", 180, degrees=True), L / 2, Wd / 2),
        ((L / 2, 0.0, Hh / 2), Rotation.from_euler("x", -90, degrees=True), L / 2, Hh / 2),
        ((L / 2, Wd, Hh / 2), Rotation.from_euler("x", 90, degrees=True), L / 2, Hh / 2),
        ((0.0, Wd / 2, Hh / 2), Rotation.from_euler("y", 90, degrees=True), Hh / 2, Wd / 2),
        ((L, Wd / 2, Hh / 2), Rotation.from_euler("y", -90, degrees=True), Hh / 2, Wd / 2),
    ]
    areas = np.array([4 * a * b for _, _, a, b in faces])
    counts = np.floor(rest * areas / areas.sum()).astype(int)
    counts[0] += rest - counts.sum()
    parts = [_free(rng, n_free, (0.3, 0.3, 0.3), (L - 0.3, Wd - 0.3, Hh - 0.3))]
    for (c, fr, a, b), m in zip(faces, counts):
        parts.append(_on_plane(rng, int(m), c, fr, a, b))
    return _concat(parts)


def _room_walk(rng, K, W, H, f):
    pos = np.array([4.0, 3.0, 1.5])
    yaw = rng.uniform(0, 2 * math.pi)
    cams = []
    for _ in range(K):
        fwd = np.array([math.cos(yaw), math.sin(yaw), 0.0])
        R, t = look_at(pos, fwd)
        cams.append(camera_array(f, f, W / 2.0, H / 2.0, R, t))
        yaw += math.radians(rng.uniform(-10.0, 10.0))
        step = 0.3 * np.array([math.cos(yaw), math.sin(yaw), 0.0])
        nxt = pos + step
        if not (0.8 < nxt[0] < 7.2 and 0.8 < nxt[1] < 5.2):
            yaw += math.pi
            nxt = pos - step
        pos = nxt
    return cams


def _smooth_texture(rng, means, waves=6, amp=0.1, cycles=(0.3, 2.5), noise=0.02):
    """Colour as a smooth function of the position: 0.5 + a sum of plane waves per channel
    (random directions, 0.3 to 2.5 cycles per metre) + a little per-Gaussian noise, clipped to
    [0, 1]. Neighbouring Gaussians then have similar colours, like a photographed surface, so
    views of the map agree with one another whatever the compositing order of close splats."""
    p = np.asarray(means, np.float64)
    out = np.full((len(p), 3), 0.5)
    for c in range(3):
        for _ in range(waves):
            d = rng.normal(size=3)
            k = d / np.linalg.norm(d) * rng.uniform(*cycles) * 2 * math.pi
            out[:, c] += amp * np.sin(p @ k + rng.uniform(0, 2 * math.pi))
    out += rng.normal(0, noise, out.shape)
    return np.clip(out, 0.0, 1.0)


def _turn(rng, K, W, H, f, degrees=90.0):
    """K views from the middle of the room turning by `degrees` of yaw in equal steps."""
    pos = np.array([4.0, 3.0, 1.5])
    yaw0 = rng.uniform(0, 2 * math.pi)
    cams = []
    for i in range(K):
        yaw = yaw0 + math.radians(degrees) * i / max(K - 1, 1)
        R, t = look_at(pos, np.array([math.cos(yaw), math.sin(yaw), 0.0]))
        cams.append(camera_array(f, f, W / 2.0, H / 2.0, R, t))
    return cams


def _aerial(rng, n):
    """Ground plane plus 40 boxes; 20% large semi-transparent Gaussians."""
    n_large = n // 5
    n_ground = (n - n_large) // 2
    n_boxes = n - n_large - n_ground
    half = 40.0
    parts = [_on_plane(rng, n_ground, (0.0, 0.0, 0.0), Rotation.identity(), half, half,
                       normal_ls=(-6.0, 0.3), inplane_ls=(-4.0, 0.7))]
    per_box = [n_boxes // 40 + (1 if i < n_boxes % 40 else 0) for i in range(40)]
    for m in per_box:
        cx_, cy_ = rng.uniform(-half + 5, half - 5, size=2)
        sx, sy = rng.uniform(2.0, 8.0, size=2)
        h = rng.uniform(2.0, 10.0)
        yaw = rng.uniform(0, 360)
        box = Rotation.from_euler("z", yaw, degrees=True)
        faces = [((0, 0, h), Rotation.identity(), sx / 2, sy / 2),
                 ((sx / 2, 0, h / 2), Rotation.from_euler("y", 90, degrees=True), h / 2, sy / 2),
                 ((-sx / 2, 0, h / 2), Rotation.from_euler("y", -90, degrees=True), h / 2, sy / 2),
                 ((0, sy / 2, h / 2), Rotation.from_euler("x", -90, degrees=True), sx / 2, h / 2),
                 ((0, -sy / 2, h / 2), Rotation.from_euler("x", 90, degrees=True), sx / 2, h / 2)]
        sub = [m // 5 + (1 if i < m % 5 else 0) for i in range(5)]
        for (c, fr, a, b), k in zip(faces, sub):
            center = box.apply(np.asarray(c, np.float64)) + np.array([cx_, cy_, 0.0])
            parts.append(_on_plane(rng, k, center, box * fr, a, b,
                                   normal_ls=(-6.0, 0.3), inplane_ls=(-4.0, 0.7)))
    large = _free(rng, n_large, (-half, -half, 0.0), (half, half, 8.0),
                  ls_mu=-2.0, ls_sd=0.5, logit_mu=-1.0, logit_sd=1.0)
    parts.append(large)
    return _concat(parts)


def _aerial_path(rng, K, W, H, f):
    cams = []
    pos = np.array([rng.uniform(-20, 20), rng.uniform(-20, 20), rng.uniform(3, 10)])
    yaw = rng.uniform(0, 2 * math.pi)
    tilt = math.radians(20.0)
    for _ in range(K):
        fwd = np.array([math.cos(yaw) * math.cos(tilt), math.sin(yaw) * math.cos(tilt), -math.sin(tilt)])
        R, t = look_at(pos, fwd)
        cams.append(camera_array(f, f, W / 2.0, H / 2.0, R, t))
        yaw += math.radians(rng.uniform(-10.0, 10.0))
        pos = pos + np.array([0.5 * math.cos(yaw), 0.5 * math.sin(yaw), rng.uniform(-0.3, 0.3)])
        pos[2] = min(10.0, max(3.0, pos[2]))
    return cams


# ----------------------------------------------------------------------------- workloads

#: name -> (default seed, N, K, W, H, f, storage dtype of the attributes)
SCENE_CONFIGS = {
    "fwd10k": (1000, 10_000, 1, 320, 240, 300.0, "f32"),
    "map100k": (1001, 100_000, 1, 640, 480, 525.0, "f32"),
    "track300k": (1002, 300_000, 1, 640, 480, 525.0, "f32"),
    "window500k": (1003, 500_000, 8, 640, 480, 525.0, "bf16"),
    "aerial2m": (1004, 2_000_000, 16, 1280, 720, 900.0, "f16"),
    "turn_room": (1005, 500_000, 10, 672, 376, 260.0, "f32"),
    "turn_room_detail": (1006, 1_000_000, 10, 672, 376, 260.0, "f32"),
}


def make_scene(name: str, seed: int | None = None, n: int | None = None, K: int | None = None,
               W: int | None = None, H: int | None = None, f: float | None = None) -> Scene:
    """Build a named workload. ``n``, ``K``, ``W``, ``H`` and ``f`` shrink it for tests.

    fwd10k     : N free Gaussians in [-2,2]^2 x [2,8], identity camera.
    map100k    : half free, half on 3 random planes; target = perturbed copy
                 (means + N(0, 1 cm), colours + N(0, 0.05)).
    track300k  : the map100k mixture; ``track_cams`` = pose perturbed by 2 deg / 5 cm.
    window500k : 6 walls of a room + 10% free; K views on a 0.3 m / +-10 deg yaw walk.
    aerial2m   : ground + 40 boxes + 20% large translucent; K views at 3-10 m, 20 deg tilt.
    turn_room  : the window500k room with a smooth colour texture; K views (672 x 376) from its
                 middle turning by 90 deg of yaw: the key-frame sequence of a robot's turn,
                 rendered from this map.
    turn_room_detail : the same turn in a denser room (1M Gaussians, splats 0.6x as wide)
                 whose texture adds a fine band (6 to 15 cycles per metre, a few pixels per cycle
                 at the turn's distances) to the smooth one: detail that key-frame insertion at a
                 4-pixel stride cannot reproduce, so reaching a PSNR takes optimisation.
    """
    dseed, dn, dK, dW, dH, df, _ = SCENE_CONFIGS[name]
    seed = dseed if seed is None else seed
    n = dn if n is None else n
    K = dK if K is None else K
    W = dW if W is None else W
    H = dH if H is None else H
    f = df if f is None else f
    rng = np.random.default_rng(seed)
    if name == "fwd10k":
        d = _free(rng, n, (-2, -2, 2), (2, 2, 8))
        cams = [identity_camera(W, H, f) for _ in range(K)]
        return _to_scene(d, cams, W, H, name)
    if name in ("map100k", "track300k"):
        d = _plane_mixture(rng, n)
        cams = [identity_camera(W, H, f) for _ in range(K)]
        s = _to_scene(d, cams, W, H, name)
        if name == "map100k":
            s.target = _perturbed_copy(rng, s)
        else:
            s.track_cams = np.stack([perturb_pose(c, rng, 2.0, 0.05) for c in s.cams])
        return s
    if name == "window500k":
        d = _room(rng, n)
        s = _to_scene(d, _room_walk(rng, K, W, H, f), W, H, name)
        s.target = _perturbed_copy(rng, s)
        return s
    if name == "turn_room":
        d = _room(rng, n)
        d["rgb"] = _smooth_texture(rng, d["means"])
        return _to_scene(d, _turn(rng, K, W, H, f), W, H, name)
    if name == "turn_room_detail":
        d = _room(rng, n)
        d["log_scales"] -= np.float32(0.5)  # finer splats than turn_room's
        d["rgb"] = np.clip(_smooth_texture(rng, d["means"]) + _smooth_texture(rng, d["means"], waves=4, amp=0.05,
                                                                               cycles=(6.0, 15.0), noise=0.0) - 0.5,
                           0.0, 1.0)
        return _to_scene(d, _turn(rng, K, W, H, f), W, H, name)
    if name == "aerial2m":
        d = _aerial(rng, n)
        s = _to_scene(d, _aerial_path(rng, K, W, H, f), W, H, name)
        s.target = _perturbed_copy(rng, s)
        s.track_cams = np.stack([perturb_pose(c, rng, 2.0, 0.05) for c in s.cams[:1]])
        return s
    raise KeyError(name)


def random_image(seed: int, shape, lo=-1.0, hi=1.0) -> np.ndarray:
    """Seeded uniform float32 array, e.g. an upstream gradient dL/dimage."""
    return np.random.default_rng(seed).uniform(lo, hi, size=shape).astype(np.float32)


def sh_coefficients(seed: int, n: int, degree: int, dc_range=1.0, rest_sd=0.15) -> np.ndarray:
    """Seeded float32 spherical-harmonic colour coefficients [n, (degree + 1)^2, 3]: the first
    (constant) triple uniform in [-dc_range, dc_range], the others normal with sd rest_sd."""
    rng = np.random.default_rng(seed)
    f = rng.normal(0.0, rest_sd, (n, (degree + 1) ** 2, 3))
    f[:, 0] = rng.uniform(-dc_range, dc_range, (n, 3))
    return f.astype(np.float32)
