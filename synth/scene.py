"""Procedural room scene and a CPU ray caster producing RGB-D frames.

The room is the axis-aligned box [0, 8] x [0, 6] x [0, 3] m (z up) holding
20 yaw-rotated boxes, each resting on the floor or floating.  Every surface
point gets an RGB colour from a per-object base colour plus a multi-octave 3D
value noise, so the quadtree seeding (Sec. III-B.2) sees a realistic mix of
flat and textured regions.  Depth is the camera-space z of the first hit,
set to 0 (invalid) outside [0.5, 6] m.

Camera convention: pixel (i, j) spans [i, i+1) x [j, j+1) with its centre at
(i + 0.5, j + 0.5); a camera-frame point (x, y, z) (x right, y down, z
forward) projects to (fx x / z + cx, fy y / z + cy).  A pose is the world to
camera transform T_CW = (R_cw, t_cw), p_c = R_cw p_w + t_cw, i.e. the inverse
of the paper's T_WC (Eq. 4).
"""
from __future__ import annotations

import dataclasses

import numpy as np

ROOM = np.array([8.0, 6.0, 3.0])
DEPTH_MIN, DEPTH_MAX = 0.5, 6.0


@dataclasses.dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int


@dataclasses.dataclass
class Pose:
    """World-to-camera rigid transform: p_c = R @ p_w + t (float32)."""

    R: np.ndarray
    t: np.ndarray

    @property
    def center(self) -> np.ndarray:
        return -(self.R.astype(np.float64).T @ self.t.astype(np.float64))


def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> Pose:
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])  # rows: camera x (right), y (down), z (forward)
    t = -R @ eye
    return Pose(R.astype(np.float32), t.astype(np.float32))


def yaw_pitch_pose(eye, yaw, pitch) -> Pose:
    fwd = np.array([np.cos(pitch) * np.cos(yaw), np.cos(pitch) * np.sin(yaw), np.sin(pitch)])
    return look_at(eye, np.asarray(eye, np.float64) + fwd)


# ----------------------------------------------------------------------------
# value noise
# ----------------------------------------------------------------------------
_M1 = np.uint64(0xFF51AFD7ED558CCD)
_M2 = np.uint64(0xC4CEB9FE1A85EC53)


def _hash3(ix, iy, iz, seed: int) -> np.ndarray:
    """Integer lattice point -> uniform [0, 1) (splitmix-style finaliser)."""
    with np.errstate(over="ignore"):
        h = (ix.astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)
             ^ iy.astype(np.uint64) * np.uint64(0xBF58476D1CE4E5B9)
             ^ iz.astype(np.uint64) * np.uint64(0x94D049BB133111EB)
             ^ np.uint64(seed) * np.uint64(0x2545F4914F6CDD1D))
        h ^= h >> np.uint64(33)
        h *= _M1
        h ^= h >> np.uint64(33)
        h *= _M2
        h ^= h >> np.uint64(33)
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 2.0**53)


def value_noise(p: np.ndarray, seed: int) -> np.ndarray:
    """Trilinear value noise with smoothstep weights, values in [0, 1)."""
    fl = np.floor(p)
    f = p - fl
    w = f * f * (3.0 - 2.0 * f)
    i = fl.astype(np.int64)
    out = np.zeros(p.shape[0])
    for dx in (0, 1):
        wx = w[:, 0] if dx else 1.0 - w[:, 0]
        for dy in (0, 1):
            wy = w[:, 1] if dy else 1.0 - w[:, 1]
            for dz in (0, 1):
                wz = w[:, 2] if dz else 1.0 - w[:, 2]
                out += wx * wy * wz * _hash3(i[:, 0] + dx, i[:, 1] + dy, i[:, 2] + dz, seed)
    return out


# ----------------------------------------------------------------------------
# room
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Room:
    box_center: np.ndarray    # [B, 3]
    box_half: np.ndarray      # [B, 3]
    box_yaw: np.ndarray       # [B]
    colors: np.ndarray        # [6 + B, 3] base colour per object (walls first)
    noise_seed: int
    noise_amp: float
    noise_freq: float
    octaves: int


def make_room(seed: int, n_boxes: int = 20, noise_amp: float = 0.5, noise_freq: float = 45.0,
              octaves: int = 3, keep_clear=()) -> Room:
    """Seeded room: 6 planes + ``n_boxes`` yaw-rotated boxes (edges 0.2-1.5 m).

    ``keep_clear`` lists points (camera centres) that no box may contain
    (with a 0.3 m margin)."""
    rng = np.random.default_rng(seed)
    centers, halves, yaws = [], [], []
    clear = [np.asarray(c, np.float64) for c in keep_clear]
    while len(centers) < n_boxes:
        half = rng.uniform(0.2, 1.5, 3) / 2.0
        yaw = rng.uniform(0.0, 2.0 * np.pi)
        xy = rng.uniform([0.3 + half.max(), 0.3 + half.max()],
                         [ROOM[0] - 0.3 - half.max(), ROOM[1] - 0.3 - half.max()])
        z0 = 0.0 if rng.uniform() < 0.5 else rng.uniform(0.3, 2.0)
        z0 = min(z0, ROOM[2] - 2.0 * half[2] - 0.05)
        c = np.array([xy[0], xy[1], z0 + half[2]])
        ok = True
        for p in clear:
            q = _to_box(p[None], c, yaw)[0]
            if np.all(np.abs(q) < half + 0.3):
                ok = False
        if ok:
            centers.append(c)
            halves.append(half)
            yaws.append(yaw)
    colors = rng.uniform(0.0, 1.0, (6 + n_boxes, 3))
    return Room(np.array(centers), np.array(halves), np.array(yaws), colors,
                int(rng.integers(1, 2**31)), noise_amp, noise_freq, octaves)


def _to_box(p, c, yaw):
    cs, sn = np.cos(yaw), np.sin(yaw)
    d = p - c
    return np.stack([cs * d[:, 0] + sn * d[:, 1], -sn * d[:, 0] + cs * d[:, 1], d[:, 2]], 1)


def _rot_dir(d, yaw):
    cs, sn = np.cos(yaw), np.sin(yaw)
    return np.stack([cs * d[:, 0] + sn * d[:, 1], -sn * d[:, 0] + cs * d[:, 1], d[:, 2]], 1)


def raycast(room: Room, cam: Camera, pose: Pose):
    """Render (rgb [H, W, 3] float32 in [0, 1], depth [H, W] float32 camera z)."""
    H, W = cam.height, cam.width
    jj, ii = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    dc = np.stack([(ii + 0.5 - cam.cx) / cam.fx, (jj + 0.5 - cam.cy) / cam.fy, np.ones_like(ii)], -1)
    dc = dc.reshape(-1, 3)
    R = pose.R.astype(np.float64)
    dw = dc @ R  # R^T applied to each row: world direction (unnormalised, camera z = 1)
    o = pose.center
    M = dw.shape[0]
    best_t = np.full(M, np.inf)
    obj = np.full(M, -1, np.int64)
    # room walls (seen from inside): for each axis the exit plane
    for ax in range(3):
        d = dw[:, ax]
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.where(d > 0, (ROOM[ax] - o[ax]) / d, np.where(d < 0, (0.0 - o[ax]) / d, np.inf))
        side = np.where(d > 0, 1, 0)
        better = (t > 0) & (t < best_t)
        best_t = np.where(better, t, best_t)
        obj = np.where(better, 2 * ax + side, obj)
    # boxes (slab test in the box frame)
    for b in range(room.box_center.shape[0]):
        ob = _to_box(o[None], room.box_center[b], room.box_yaw[b])[0]
        db = _rot_dir(dw, room.box_yaw[b])
        hb = room.box_half[b]
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / db
            t1 = (-hb[None] - ob[None]) * inv
            t2 = (hb[None] - ob[None]) * inv
        tmin = np.nanmax(np.minimum(t1, t2), axis=1)
        tmax = np.nanmin(np.maximum(t1, t2), axis=1)
        hit = (tmax >= tmin) & (tmin > 0)
        better = hit & (tmin < best_t)
        best_t = np.where(better, tmin, best_t)
        obj = np.where(better, 6 + b, obj)
    p = o[None] + best_t[:, None] * dw
    depth = best_t  # camera z of the hit (direction has camera z = 1)
    base = room.colors[obj]
    noise = np.zeros_like(base)
    amp = 1.0
    for k in range(room.octaves):
        f = room.noise_freq * (2.0 ** k)
        for ch in range(3):
            noise[:, ch] += amp * (value_noise(p * f, room.noise_seed + 101 * k + 7 * ch) - 0.5) * 2.0
        amp *= 0.5
    rgb = np.clip(base + room.noise_amp * noise, 0.0, 1.0)
    depth = np.where((depth >= DEPTH_MIN) & (depth <= DEPTH_MAX), depth, 0.0)
    return rgb.reshape(H, W, 3).astype(np.float32), depth.reshape(H, W).astype(np.float32)
