"""Workload recipes (seed = 1000 + recipe index).

``tiny_random``   64x48 px, fx=fy=60, identity pose, 500 random Gaussians in
                  the view frustum (uniform in volume at depth 0.5-4 m),
                  log-scales U[-4, -1], random unit quaternions, opacity
                  logits N(0, 1), SH degree 0 with decoded RGB U[0, 1];
                  target RGB U[0, 1] and target depth U[0.5, 4] per pixel.
``single_view``   1200x680, fx=fy=600: one synthetic room frame, quadtree
                  seeded (about 300k Gaussians), SH degree 3; the frame itself
                  is the target.
``scale_stress``  1752x1168, fx=fy=1200: exactly 1M quadtree-seeded
                  Gaussians, 20% of them replaced by large ones (log-scale
                  U[-1, 0], opacity logit +2).
``multi_view``    8 uneven views (2x 640x480 fx=320, 4x 1200x680 fx=600,
                  2x 1752x1168 fx=1200) within 2 m and +-30 deg of the room
                  centre, sharing one 500k-Gaussian map seeded from all views
                  with a one-Gaussian-per-voxel novelty rule.

All arrays are float32 numpy; images are planar ([3, H, W] and [H, W]).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .quadtree import Y00, seed_gaussians
from .scene import Camera, Pose, look_at, make_room, raycast, yaw_pitch_pose

ROOM_CENTER = np.array([4.0, 3.0, 1.5])


@dataclasses.dataclass
class View:
    cam: Camera
    pose: Pose
    target_rgb: np.ndarray   # [3, H, W]
    target_depth: np.ndarray  # [H, W]


@dataclasses.dataclass
class Workload:
    name: str
    params: dict
    views: list

    @property
    def n(self) -> int:
        return int(self.params["means"].shape[0])

    @property
    def sh_degree(self) -> int:
        return int(self.params["sh_degree"])


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    return (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)


def random_gaussians(rng, n, cam: Camera, pose: Pose, sh_degree=0, z_range=(0.5, 4.0),
                     log_scale_range=(-4.0, -1.0), sh_rest_std=0.0):
    """Gaussians uniform in volume inside the frustum of (cam, pose)."""
    a, b = z_range
    z = (a**3 + rng.uniform(0, 1, n) * (b**3 - a**3)) ** (1.0 / 3.0)
    u = rng.uniform(0, cam.width, n)
    v = rng.uniform(0, cam.height, n)
    pc = np.stack([(u - cam.cx) * z / cam.fx, (v - cam.cy) * z / cam.fy, z], 1)
    pw = (pc - pose.t.astype(np.float64)[None]) @ pose.R.astype(np.float64)
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n, K, 3), np.float32)
    sh[:, 0, :] = (rng.uniform(0, 1, (n, 3)) - 0.5) / Y00
    if K > 1 and sh_rest_std > 0:
        sh[:, 1:, :] = rng.normal(0.0, sh_rest_std, (n, K - 1, 3))
    return {
        "means": pw.astype(np.float32),
        "log_scales": rng.uniform(*log_scale_range, (n, 3)).astype(np.float32),
        "quats": _unit_quats(rng, n),
        "opacity_logits": rng.standard_normal(n).astype(np.float32),
        "sh": sh,
        "sh_degree": sh_degree,
    }


def tiny_random(seed: int = 1000, n: int = 500, width: int = 64, height: int = 48, f: float = 60.0,
                sh_degree: int = 0, sh_rest_std: float = 0.0) -> Workload:
    rng = np.random.default_rng(seed)
    cam = Camera(f, f, width / 2.0, height / 2.0, width, height)
    pose = Pose(np.eye(3, dtype=np.float32), np.zeros(3, np.float32))
    params = random_gaussians(rng, n, cam, pose, sh_degree, sh_rest_std=sh_rest_std)
    trgb = rng.uniform(0, 1, (3, height, width)).astype(np.float32)
    tdep = rng.uniform(0.5, 4.0, (height, width)).astype(np.float32)
    return Workload("tiny_random", params, [View(cam, pose, trgb, tdep)])


# three small views of uneven size around one cloud of random Gaussians
TINY_MULTI_CAMS = ((64, 48, 60.0), (40, 24, 40.0), (72, 56, 70.0))
TINY_MULTI_EYES = ((0.0, 0.0, 0.0), (0.3, -0.4, 0.15), (-0.2, 0.35, -0.2))
TINY_MULTI_TARGET = (2.5, 0.0, 0.0)


def tiny_multi_view(seed: int = 1004, n: int = 500, sh_degree: int = 0, sh_rest_std: float = 0.0,
                    cams=TINY_MULTI_CAMS) -> Workload:
    """Views of uneven resolution looking at one cloud of random Gaussians
    (placed in the frustum of the first view, 1.5-3.5 m away); targets are
    uniform random images as in tiny_random."""
    rng = np.random.default_rng(seed)
    views = []
    for k, (w, h, f) in enumerate(cams):
        cam = Camera(f, f, w / 2.0, h / 2.0, w, h)
        pose = look_at(np.asarray(TINY_MULTI_EYES[k % len(TINY_MULTI_EYES)]) * (1 + k // len(TINY_MULTI_EYES)),
                       TINY_MULTI_TARGET)
        views.append(View(cam, pose, rng.uniform(0, 1, (3, h, w)).astype(np.float32),
                          rng.uniform(0.5, 4.0, (h, w)).astype(np.float32)))
    params = random_gaussians(rng, n, views[0].cam, views[0].pose, sh_degree, z_range=(1.5, 3.5),
                              sh_rest_std=sh_rest_std)
    return Workload("tiny_multi_view", params, views)


def _frame(room, cam, pose):
    rgb, depth = raycast(room, cam, pose)
    return rgb, depth


SINGLE_VIEW_EYE = np.array([3.2, 2.6, 1.4])
SINGLE_VIEW_TARGET = np.array([8.0, 4.8, 0.9])


def single_view(seed: int = 1001, width: int = 1200, height: int = 680, f: float = 600.0,
                sh_degree: int = 3, sh_rest_std: float = 0.0) -> Workload:
    """One room frame, quadtree seeded; the frame is the optimisation target."""
    cam = Camera(f, f, width / 2.0, height / 2.0, width, height)
    pose = look_at(SINGLE_VIEW_EYE, SINGLE_VIEW_TARGET)
    room = make_room(seed, keep_clear=[SINGLE_VIEW_EYE])
    rgb, depth = _frame(room, cam, pose)
    params = seed_gaussians(rgb, depth, cam, pose, sh_degree)
    if sh_rest_std > 0 and sh_degree > 0:
        rng = np.random.default_rng(seed + 7)
        params["sh"][:, 1:, :] = rng.normal(0.0, sh_rest_std, params["sh"][:, 1:, :].shape)
    view = View(cam, pose, np.ascontiguousarray(rgb.transpose(2, 0, 1)), depth)
    return Workload("single_view", params, [view])


def _resize(params: dict, n: int, rng, cam: Camera, pose: Pose, rgb, depth) -> dict:
    """Seeded subsample (or pad with 1-px-leaf Gaussians at random pixels) to exactly n."""
    m = params["means"].shape[0]
    if m >= n:
        idx = np.sort(rng.choice(m, n, replace=False))
        return {k: (v[idx] if isinstance(v, np.ndarray) else v) for k, v in params.items()}
    extra = n - m
    ok = np.argwhere(depth > 0)
    pick = ok[rng.integers(0, ok.shape[0], extra)]
    pj, pi = pick[:, 0], pick[:, 1]
    z = depth[pj, pi].astype(np.float64)
    uc, vc = pi + rng.uniform(0, 1, extra), pj + rng.uniform(0, 1, extra)
    pc = np.stack([(uc - cam.cx) * z / cam.fx, (vc - cam.cy) * z / cam.fy, z], 1)
    pw = (pc - pose.t.astype(np.float64)[None]) @ pose.R.astype(np.float64)
    d = 0.5 * np.sqrt(2.0) * z / cam.fx
    K = params["sh"].shape[1]
    sh = np.zeros((extra, K, 3), np.float32)
    sh[:, 0, :] = (rgb[pj, pi] - 0.5) / Y00
    q = np.zeros((extra, 4), np.float32)
    q[:, 0] = 1
    add = {"means": pw.astype(np.float32), "log_scales": np.repeat(np.log(d)[:, None], 3, 1).astype(np.float32),
           "quats": q, "opacity_logits": np.zeros(extra, np.float32), "sh": sh}
    out = dict(params)
    for k, v in add.items():
        out[k] = np.concatenate([params[k], v])
    return out


def scale_stress(seed: int = 1002, n: int = 1_000_000, width: int = 1752, height: int = 1168,
                 f: float = 1200.0, large_frac: float = 0.2) -> Workload:
    cam = Camera(f, f, width / 2.0, height / 2.0, width, height)
    pose = look_at(SINGLE_VIEW_EYE, SINGLE_VIEW_TARGET)
    room = make_room(seed, keep_clear=[SINGLE_VIEW_EYE])
    rgb, depth = _frame(room, cam, pose)
    rng = np.random.default_rng(seed + 1)
    params = _resize(seed_gaussians(rgb, depth, cam, pose, 3), n, rng, cam, pose, rgb, depth)
    big = rng.choice(n, int(round(large_frac * n)), replace=False)
    params["log_scales"][big] = rng.uniform(-1.0, 0.0, (big.size, 3)).astype(np.float32)
    params["opacity_logits"][big] = 2.0
    params["quats"][big] = _unit_quats(rng, big.size)
    view = View(cam, pose, np.ascontiguousarray(rgb.transpose(2, 0, 1)), depth)
    return Workload("scale_stress", params, [view])


MULTI_VIEW_CAMS = [(640, 480, 320.0)] * 2 + [(1200, 680, 600.0)] * 4 + [(1752, 1168, 1200.0)] * 2


def multi_view_poses(rng, n_views: int):
    poses = []
    for _ in range(n_views):
        while True:
            off = rng.uniform(-2.0, 2.0, 3)
            if np.linalg.norm(off) <= 2.0:
                break
        eye = ROOM_CENTER + off
        eye = np.clip(eye, [0.4, 0.4, 0.4], [7.6, 5.6, 2.6])
        yaw = np.deg2rad(rng.uniform(-30.0, 30.0))
        pitch = np.deg2rad(rng.uniform(-30.0, 30.0))
        poses.append((eye, yaw, pitch))
    return poses


def _multi_view_frame(args):
    """One view of the multi-view set: ray-cast frame and its seeded
    Gaussians (a process-pool worker; the room is rebuilt from its seed)."""
    seed, keep_clear, (w, h, f), (eye, yaw, pitch) = args
    room = make_room(seed, keep_clear=keep_clear)
    cam = Camera(f, f, w / 2.0, h / 2.0, w, h)
    pose = yaw_pitch_pose(eye, yaw, pitch)
    rgb, depth = _frame(room, cam, pose)
    return cam, pose, rgb, depth, seed_gaussians(rgb, depth, cam, pose, 3)


def multi_view(seed: int = 1003, n: int = 500_000, voxel: float = 0.01, cams=None, workers: int = 1) -> Workload:
    """Uneven views sharing one map; seeding keeps at most one Gaussian per voxel
    (the paper's TSDF-weight novelty check, Sec. III-B.2, reduced to voxel
    occupancy since no TSDF map is built here).  ``workers`` > 1 ray-casts and
    seeds the views in a spawned process pool (same result)."""
    rng = np.random.default_rng(seed)
    cams = cams or MULTI_VIEW_CAMS
    specs = multi_view_poses(rng, len(cams))
    keep_clear = [s[0] for s in specs]
    jobs = [(seed, keep_clear, c, sp) for c, sp in zip(cams, specs)]
    if workers > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, len(jobs))) as pool:
            frames = pool.map(_multi_view_frame, jobs)
    else:
        frames = [_multi_view_frame(j) for j in jobs]
    views, parts = [], []
    seen = set()
    for cam, pose, rgb, depth, p in frames:
        vox = np.floor(p["means"].astype(np.float64) / voxel).astype(np.int64)
        keys = (vox[:, 0] * 1_000_003 + vox[:, 1]) * 1_000_033 + vox[:, 2]
        _, first = np.unique(keys, return_index=True)
        keep = np.zeros(keys.shape[0], bool)
        keep[first] = True
        for i in np.flatnonzero(keep):
            if keys[i] in seen:
                keep[i] = False
        seen.update(keys[keep].tolist())
        parts.append({k: (v[keep] if isinstance(v, np.ndarray) else v) for k, v in p.items()})
        views.append(View(cam, pose, np.ascontiguousarray(rgb.transpose(2, 0, 1)), depth))
    params = {k: np.concatenate([q[k] for q in parts]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    params["sh_degree"] = 3
    big_view = views[-1]
    rgb_last = big_view.target_rgb.transpose(1, 2, 0)
    params = _resize(params, n, rng, big_view.cam, big_view.pose, rgb_last, big_view.target_depth)
    return Workload("multi_view", params, views)


RECIPES = {
    "tiny_random": tiny_random,
    "single_view": single_view,
    "scale_stress": scale_stress,
    "multi_view": multi_view,
}


# ----------------------------------------------------------------------------
# streaming per-frame sequence
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Stream:
    """A smooth camera trajectory through one synthetic room; ``frame(k)``
    ray-casts frame k (RGB [H, W, 3] and depth [H, W], float32)."""
    room: object
    cam: Camera
    poses: list

    def frame(self, k: int):
        return raycast(self.room, self.cam, self.poses[k])


def stream_poses(n_frames: int, radius=(1.6, 1.1), height=0.25, sweep=np.pi):
    """Eye on an ellipse around the room centre (half a turn over the
    sequence by default), looking across the room (inwards, with a slow yaw
    swing) and a slow pitch oscillation."""
    poses, eyes = [], []
    for k in range(n_frames):
        s = k / max(n_frames - 1, 1)
        a = sweep * s
        eye = ROOM_CENTER + np.array([radius[0] * np.cos(a), radius[1] * np.sin(a), height * np.sin(2 * a) - 0.1])
        yaw = a + np.pi + 0.5 * np.sin(3 * a)
        pitch = -0.12 + 0.1 * np.sin(2 * np.pi * s)
        poses.append(yaw_pitch_pose(eye, yaw, pitch))
        eyes.append(eye)
    return poses, eyes


def streaming(seed: int = 1005, n_frames: int = 200, width: int = 1200, height: int = 680, f: float = 600.0) -> Stream:
    """The per-frame streaming sequence: ``n_frames`` frames of a smooth
    trajectory through a room generated with the trajectory kept clear of
    boxes."""
    poses, eyes = stream_poses(n_frames)
    room = make_room(seed, keep_clear=eyes[:: max(1, n_frames // 40)] + [eyes[-1]])
    cam = Camera(f, f, width / 2.0, height / 2.0, width, height)
    return Stream(room, cam, poses)
