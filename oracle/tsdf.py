"""FP64 reference of the TSDF fusion (Sec. III-B.1, Eq. 6-9) and of the
voxel-weight novelty check that gates the per-frame seeding (Sec. III-B.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The map is a single-resolution TSDF grid of voxels of side ``s``, stored as
blocks of 8^3 voxels (the leaf blocks of the octree of Sec. III-A.1); here a
block is a dict entry keyed by its integer block coordinates, holding the
tsdf and weight of its voxels as float64 arrays indexed [z, y, x].  Voxel
(gx, gy, gz) has its centre at ((g + 0.5) s) and lies in block floor(g / 8).

Definition followed, with the readings where the paper is silent:

* Allocation (Sec. III-B.1): for every pixel (i, j) with a finite depth
  D > 0, the ray through the pixel centre (i + 0.5, j + 0.5) is sampled at
  the camera depths z_k = D + c_k, c_k = -eps + k (2 eps / n), k = 0..n,
  n = ceil(eps / (2 s)) (sample spacing at most half a block along the
  depth; samples with z <= 0 are dropped); every block holding a sample
  (block coordinates in [-2^20, 2^20)) is allocated and is "touched" by the
  frame.  Only touched blocks are integrated.
* Integration (Eq. 6-9), for every voxel of a touched block: camera point
  p_c = R p_v + t of its centre (world-to-camera pose R, t); skipped if
  z <= 0, if pi(p_c) = (fx x/z + cx, fy y/z + cy) falls outside the image,
  if the depth D at pixel floor(pi(p_c)) is not > 0, or if
  sdf = D - z < -eps (the truncation region behind the surface, where
  KinectFusion, whose integration the paper says it follows, stores no
  measurement).  Otherwise tsdf = min(1, sdf/eps) for sdf > 0 and
  max(-1, sdf/eps) else (Eq. 7), w_k = min(w_max, w_{k-1} + 1) (Eq. 8) and
  Eq. 9 as printed: tsdf_k = (tsdf_{k-1} w_{k-1} + tsdf w_k) / (w_{k-1} + w_k).
  ``fusion="unit"`` instead weights the new measurement by 1, as in
  KinectFusion: (tsdf_{k-1} w_{k-1} + tsdf) / (w_{k-1} + 1).
* Every quantity is evaluated in float64 on the float32 values the kernels
  receive (depth image, pose, intrinsics, voxel size, truncation): the
  integer decisions (the block of a sample, the pixel of a voxel, whether it
  is updated, the voxel of p_q) are those of the exact arithmetic, up to
  float64 rounding.  Where a float32 implementation may decide the other way
  (a value within its rounding error of a boundary), the oracle reports how
  far the float64 value lies from the boundary: ``allocation_samples`` gives
  every sample's block coordinates as reals, every voxel keeps the smallest
  distance of its projection to a pixel edge or the image border (pixels)
  and of its sdf to -eps (metres) over the frames that reached it, and
  ``leaf_points`` gives each Eq. 10 point's distance to a voxel face.
* Novelty (Sec. III-B.2): a quadtree leaf whose Eq. 10 point p_q lies in a voxel of weight exactly 1 after this
  frame's integration is new; a voxel of a block that is not allocated
  counts as weight 0 (not new).  A voxel holds at most one Gaussian
  (Sec. IV-C.1): among the new leaves that fall in one voxel, the one whose
  top-left pixel has the smallest row-major index y0 W + x0 seeds it.
"""
from __future__ import annotations

import math

import numpy as np

from . import quadtree as _qt

BLOCK = 8
F32 = np.float32


def n_band_steps(eps: float, voxel_size: float) -> int:
    """n of the band samples: spacing 2 eps / n at most half a block."""
    return max(1, int(math.ceil(float(F32(eps)) / (2.0 * float(F32(voxel_size))) - 1e-6)))


def band_offsets(eps: float, voxel_size: float) -> np.ndarray:
    """c_k = -eps + k 2 eps / n, float64."""
    e = float(F32(eps))
    n = n_band_steps(eps, voxel_size)
    return np.array([-e + k * (2.0 * e / n) for k in range(n + 1)], np.float64)


def _pose64(R, t):
    """The pose as the kernels receive it (float32 values), in float64."""
    return (np.asarray(R, np.float64).astype(F32).astype(np.float64),
            np.asarray(t, np.float64).astype(F32).astype(np.float64))


def _cam64(cam):
    return tuple(float(F32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))


def allocation_samples(depth: np.ndarray, cam, R_cw, t_cw, voxel_size: float, eps: float) -> np.ndarray:
    """World coordinates, in block units (metres / (8 s)), of every band
    sample of every pixel with depth > 0: float64 [M, 3]."""
    R, t = _pose64(R_cw, t_cw)
    fx, fy, cx, cy = _cam64(cam)
    bs = BLOCK * float(F32(voxel_size))
    dep = np.asarray(depth, F32)
    jj, ii = np.nonzero((dep > F32(0)) & np.isfinite(dep))
    D = dep[jj, ii].astype(np.float64)
    xn = ((ii + 0.5) - cx) / fx
    yn = ((jj + 0.5) - cy) / fy
    out = []
    for ck in band_offsets(eps, voxel_size):
        z = D + ck
        ok = z > 0
        pc = np.stack([xn[ok] * z[ok], yn[ok] * z[ok], z[ok]], -1)
        out.append(((pc - t) @ R) / bs)  # R^T (p_c - t), row form
    return np.concatenate(out) if out else np.zeros((0, 3))


def blocks_of(F: np.ndarray) -> set:
    f = np.floor(F)
    inside = (np.abs(f) < 2 ** 20).all(1)  # block coordinates in [-2^20, 2^20)
    return set(map(tuple, f[inside].astype(np.int64).tolist()))


def allocate(depth: np.ndarray, cam, R_cw, t_cw, voxel_size: float, eps: float) -> set:
    """Blocks holding a band sample of some pixel's ray."""
    return blocks_of(allocation_samples(depth, cam, R_cw, t_cw, voxel_size, eps))


def block_distance(F: np.ndarray, b) -> float:
    """Smallest L-infinity distance (block units) from a sample to block b's
    box [b, b + 1)^3; 0 if a sample lies in it."""
    d = np.maximum(np.asarray(b, np.float64) - F, F - (np.asarray(b, np.float64) + 1.0))
    return float(np.maximum(d, 0.0).max(1).min()) if len(F) else math.inf


def block_depth(F: np.ndarray, b) -> float:
    """How deep (block units, L-infinity) the deepest sample lies inside block
    b: the distance it would have to move to leave it (0 if none is inside)."""
    bb = np.asarray(b, np.float64)
    m = np.minimum(F - bb, bb + 1.0 - F).min(1)
    return float(m.max(initial=0.0))


def new_block():
    """tsdf, weight, smallest pixel-edge distance (px), smallest sdf + eps
    distance (m) of the block's voxels, indexed [z, y, x]."""
    return [np.zeros((BLOCK,) * 3), np.zeros((BLOCK,) * 3), np.full((BLOCK,) * 3, np.inf),
            np.full((BLOCK,) * 3, np.inf)]


def _local_grid():
    lz, ly, lx = np.meshgrid(np.arange(BLOCK), np.arange(BLOCK), np.arange(BLOCK), indexing="ij")
    return lx.ravel(), ly.ravel(), lz.ravel()


def integrate_blocks(grid: dict, blocks, depth: np.ndarray, cam, R_cw, t_cw, voxel_size: float, eps: float,
                     w_max: float, fusion: str = "printed") -> None:
    """Eq. 6-9 on every voxel of ``blocks`` (allocated in ``grid`` if new)."""
    blocks = [tuple(int(c) for c in b) for b in blocks]
    if not blocks:
        return
    H, W = depth.shape
    R, t = _pose64(R_cw, t_cw)
    fx, fy, cx, cy = _cam64(cam)
    s = float(F32(voxel_size))
    e = float(F32(eps))
    dep = np.asarray(depth, F32)
    lx, ly, lz = _local_grid()
    B = np.array(blocks, np.int64)  # [nb, 3]
    pv = [(BLOCK * B[:, a:a + 1] + l[None, :] + 0.5) * s for a, l in enumerate((lx, ly, lz))]  # [nb, 512]
    pc = [R[r, 0] * pv[0] + R[r, 1] * pv[1] + R[r, 2] * pv[2] + t[r] for r in range(3)]
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        u = fx * (pc[0] / pc[2]) + cx
        v = fy * (pc[1] / pc[2]) + cy
    front = pc[2] > 0
    ok = front & (u >= 0) & (u < W) & (v >= 0) & (v < H)
    pi = np.where(ok, np.floor(np.where(ok, u, 0)), 0).astype(np.int64)
    pj = np.where(ok, np.floor(np.where(ok, v, 0)), 0).astype(np.int64)
    D = dep[pj, pi].astype(np.float64)
    sdf = D - pc[2]
    upd = ok & (D > 0) & (sdf >= -e)
    tsdf = np.where(sdf > 0, np.minimum(1.0, sdf / e), np.maximum(-1.0, sdf / e))
    # distances to the decision boundaries (where a float32 evaluation may
    # decide the other way): pixel edges and image border, sdf = -eps
    with np.errstate(invalid="ignore"):
        mpx = np.minimum(np.abs(u - np.round(u)), np.abs(v - np.round(v)))
        mpx = np.minimum(mpx, np.minimum(np.minimum(np.abs(u), np.abs(u - W)), np.minimum(np.abs(v), np.abs(v - H))))
    mpx = np.where(front, np.nan_to_num(mpx, nan=np.inf), np.inf)
    msdf = np.where(ok & (D > 0), np.abs(sdf + e), np.inf)
    msdf = np.minimum(msdf, np.abs(pc[2]))  # z = 0 (never near in practice)
    for n, b in enumerate(blocks):
        cell = grid.setdefault(b, new_block())
        cell[2][lz, ly, lx] = np.minimum(cell[2][lz, ly, lx], mpx[n])
        cell[3][lz, ly, lx] = np.minimum(cell[3][lz, ly, lx], msdf[n])
        m = upd[n]
        zi, yi, xi = lz[m], ly[m], lx[m]
        t_old = cell[0][zi, yi, xi]
        w_old = cell[1][zi, yi, xi]
        w_new = np.minimum(float(w_max), w_old + 1.0)
        if fusion == "printed":
            t_new = (t_old * w_old + tsdf[n][m] * w_new) / (w_old + w_new)
        elif fusion == "unit":
            t_new = (t_old * w_old + tsdf[n][m]) / (w_old + 1.0)
        else:
            raise ValueError(fusion)
        cell[0][zi, yi, xi] = t_new
        cell[1][zi, yi, xi] = w_new


def integrate(grid: dict, depth, cam, R_cw, t_cw, voxel_size: float = 0.01, eps: float = 0.08,
              w_max: float = 100.0, fusion: str = "printed") -> set:
    """One frame: allocation, then Eq. 6-9 over the touched blocks."""
    blocks = allocate(depth, cam, R_cw, t_cw, voxel_size, eps)
    integrate_blocks(grid, sorted(blocks), depth, cam, R_cw, t_cw, voxel_size, eps, w_max, fusion)
    return blocks


def leaf_points(depth, lv, cam, R_cw, t_cw):
    """Eq. 10 world points of the leaves with depth > 0 at their centre pixel;
    returns (indices into lv, points [k, 3] float64)."""
    H, W = depth.shape
    R, t = _pose64(R_cw, t_cw)
    fx, fy, cx, cy = _cam64(cam)
    lv = np.asarray(lv, np.int64).reshape(-1, 4)
    ux = lv[:, 0] + lv[:, 2] / 2.0
    uy = lv[:, 1] + lv[:, 3] / 2.0
    pi = np.minimum(np.floor(ux).astype(np.int64), W - 1)
    pj = np.minimum(np.floor(uy).astype(np.int64), H - 1)
    z = np.asarray(depth, F32)[pj, pi].astype(np.float64) if len(lv) else np.zeros(0)
    keep = np.nonzero(z > 0)[0]
    z = z[keep]
    q = np.stack([(ux[keep] - cx) * z / fx, (uy[keep] - cy) * z / fy, z], -1) - t
    return keep.astype(np.int64), (q @ R).reshape(-1, 3)


def voxel_of(points: np.ndarray, voxel_size: float):
    """Voxel index of each point and the point's distance (m) to the nearest
    voxel face (where a float32 evaluation may pick the neighbour)."""
    s = float(F32(voxel_size))
    f = np.asarray(points, np.float64) / s
    vox = np.floor(f).astype(np.int64)
    margin = (np.minimum(f - vox, vox + 1.0 - f).min(1) if len(f) else np.zeros(0)) * s
    return vox, margin


def voxel_weight(grid: dict, vox) -> float:
    """Weight of voxel ``vox`` (global integer coordinates); 0 if unallocated."""
    return float(voxel_state(grid, vox)[1])


def voxel_state(grid: dict, vox):
    """(tsdf, weight, pixel margin, sdf margin) of voxel ``vox``; weight 0 and
    infinite margins if its block is not allocated."""
    b = tuple(int(v) // BLOCK for v in vox)
    cell = grid.get(b)
    if cell is None:
        return 0.0, 0.0, math.inf, math.inf
    lx, ly, lz = (int(v) - BLOCK * bb for v, bb in zip(vox, b))
    return tuple(float(c[lz, ly, lx]) for c in cell)


def novelty(grid: dict, depth, lv, cam, R_cw, t_cw, voxel_size: float = 0.01) -> dict:
    """Per leaf with depth > 0 at its centre (``leaf``: indices into lv): its
    Eq. 10 point, voxel, the voxel's weight, the point's distance to a voxel
    face (m), the voxel's running pixel / sdf margins, and whether it seeds
    (weight exactly 1 and the smallest y0 W + x0 of its voxel's new leaves)."""
    W = depth.shape[1]
    idx, pts = leaf_points(depth, lv, cam, R_cw, t_cw)
    vox, vmargin = voxel_of(pts, voxel_size)
    st = np.array([voxel_state(grid, v) for v in vox.tolist()], np.float64).reshape(-1, 4)
    new = st[:, 1] == 1.0
    best = {}
    for k in np.nonzero(new)[0].tolist():
        n = int(idx[k])
        key = int(lv[n][1]) * W + int(lv[n][0])
        v = tuple(vox[k].tolist())
        if v not in best or key < best[v][0]:
            best[v] = (key, k)
    seeds = np.zeros(len(idx), bool)
    seeds[[k for _, k in best.values()]] = True
    return {"leaf": idx, "points": pts, "voxel": vox, "weight": st[:, 1], "voxel_margin": vmargin,
            "px_margin": st[:, 2], "sdf_margin": st[:, 3], "seeds": seeds}


def novel_leaves(grid: dict, depth, lv, cam, R_cw, t_cw, voxel_size: float = 0.01):
    """Indices into ``lv`` of the leaves that seed: Eq. 10 point in a voxel
    of weight 1, at most one (smallest y0 W + x0) per voxel."""
    r = novelty(grid, depth, lv, cam, R_cw, t_cw, voxel_size)
    return np.sort(r["leaf"][r["seeds"]])


def seed_tsdf(rgb, depth, grid: dict, cam, R_cw, t_cw, sh_degree: int, var_thr: float = 0.01, max_size: int = 64,
              min_size: int = 1, voxel_size: float = 0.01) -> dict:
    """Quadtree of the frame, the novelty check against the integrated grid,
    then Eq. 10 for the leaves that seed."""
    lv = _qt.leaves(np.asarray(rgb, np.float64), var_thr, max_size, min_size)
    sel = novel_leaves(grid, depth, lv, cam, R_cw, t_cw, voxel_size)
    R, t = _pose64(R_cw, t_cw)
    return _qt.seed(rgb, depth, lv[sel], cam, R, t, sh_degree)
