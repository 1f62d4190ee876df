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
* The integer decisions (which block a sample falls in, which pixel a voxel
  projects to, whether it is updated, which voxel p_q falls in) are taken in
  float32 with a fixed order of correctly rounded operations, the precision
  of the kernels: the same decisions on both sides.  The tsdf values are
  float64.
* Novelty (Sec. III-B.2): a quadtree leaf whose Eq. 10 point p_q (float32,
  fixed operation order) lies in a voxel of weight exactly 1 after this
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
    """c_k = -eps + k 2 eps / n (computed in float64, stored as float32)."""
    e = float(F32(eps))
    n = n_band_steps(eps, voxel_size)
    return np.array([-e + k * (2.0 * e / n) for k in range(n + 1)], np.float64).astype(F32)


def _f32_pose(R, t):
    return np.asarray(R, np.float64).astype(F32), np.asarray(t, np.float64).astype(F32)


def allocate(depth: np.ndarray, cam, R_cw, t_cw, voxel_size: float, eps: float) -> set:
    """Blocks holding a band sample of some pixel's ray (float32 decisions)."""
    H, W = depth.shape
    R, t = _f32_pose(R_cw, t_cw)
    fx, fy, cx, cy = (F32(cam.fx), F32(cam.fy), F32(cam.cx), F32(cam.cy))
    bs = F32(F32(BLOCK) * F32(voxel_size))
    dep = np.asarray(depth, F32)
    jj, ii = np.nonzero((dep > F32(0)) & np.isfinite(dep))
    D = dep[jj, ii]
    xn = ((ii.astype(F32) + F32(0.5)) - cx) / fx
    yn = ((jj.astype(F32) + F32(0.5)) - cy) / fy
    out = set()
    for ck in band_offsets(eps, voxel_size):
        z = D + ck
        ok = z > F32(0)
        pc = (xn[ok] * z[ok], yn[ok] * z[ok], z[ok])
        d = [pc[r] - t[r] for r in range(3)]
        blk = []
        inside = np.ones(d[0].shape, bool)
        for a in range(3):
            pw = (R[0, a] * d[0] + R[1, a] * d[1]) + R[2, a] * d[2]
            f = np.floor(pw / bs)
            inside &= np.abs(f) < 2 ** 20  # block coordinates in [-2^20, 2^20)
            blk.append(np.where(inside, f, 0).astype(np.int64))
        out.update(zip(blk[0][inside].tolist(), blk[1][inside].tolist(), blk[2][inside].tolist()))
    return out


def new_block():
    return [np.zeros((BLOCK,) * 3), np.zeros((BLOCK,) * 3)]


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
    R, t = _f32_pose(R_cw, t_cw)
    R64, t64 = R.astype(np.float64), t.astype(np.float64)
    fx, fy, cx, cy = (F32(cam.fx), F32(cam.fy), F32(cam.cx), F32(cam.cy))
    s = F32(voxel_size)
    e32 = F32(eps)
    e = float(e32)
    dep = np.asarray(depth, F32)
    lx, ly, lz = _local_grid()
    B = np.array(blocks, np.int64)  # [nb, 3]
    g = [BLOCK * B[:, a:a + 1] + l[None, :] for a, l in enumerate((lx, ly, lz))]  # [nb, 512] each
    pv = [(ga.astype(F32) + F32(0.5)) * s for ga in g]
    pc = [((R[r, 0] * pv[0] + R[r, 1] * pv[1]) + R[r, 2] * pv[2]) + t[r] for r in range(3)]
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        u = fx * (pc[0] / pc[2]) + cx
        v = fy * (pc[1] / pc[2]) + cy
    ok = (pc[2] > F32(0)) & (u >= F32(0)) & (u < F32(W)) & (v >= F32(0)) & (v < F32(H))
    pi = np.where(ok, np.floor(np.where(ok, u, 0)), 0).astype(np.int64)
    pj = np.where(ok, np.floor(np.where(ok, v, 0)), 0).astype(np.int64)
    D32 = dep[pj, pi]
    upd = ok & (D32 > F32(0)) & ((D32 - pc[2]) >= -e32)
    pv64 = [(ga.astype(np.float64) + 0.5) * float(s) for ga in g]
    z64 = R64[2, 0] * pv64[0] + R64[2, 1] * pv64[1] + R64[2, 2] * pv64[2] + t64[2]
    sdf = D32.astype(np.float64) - z64
    tsdf = np.where(sdf > 0, np.minimum(1.0, sdf / e), np.maximum(-1.0, sdf / e))
    for n, b in enumerate(blocks):
        cell = grid.setdefault(b, new_block())
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
    """Eq. 10 world points of the leaves with depth > 0 at their centre pixel,
    in float32 with a fixed order of correctly rounded operations (the
    precision the novelty decision is taken in); returns (indices into lv,
    points [k, 3] as float64 holding the float32 values)."""
    H, W = depth.shape
    R, t = _f32_pose(R_cw, t_cw)
    fx, fy, cx, cy = (F32(cam.fx), F32(cam.fy), F32(cam.cx), F32(cam.cy))
    idx, pts = [], []
    for n, (x0, y0, w, h) in enumerate(np.asarray(lv, np.int64)):
        ux, uy = F32(x0 + w / 2.0), F32(y0 + h / 2.0)  # exact
        pi, pj = min(int(np.floor(ux)), W - 1), min(int(np.floor(uy)), H - 1)
        z = F32(depth[pj, pi])
        if not z > 0:
            continue
        q = [((ux - cx) * z) / fx - t[0], ((uy - cy) * z) / fy - t[1], z - t[2]]
        pts.append([(R[0, a] * q[0] + R[1, a] * q[1]) + R[2, a] * q[2] for a in range(3)])
        idx.append(n)
    return np.array(idx, np.int64), np.array(pts, np.float32).astype(np.float64).reshape(-1, 3)


def voxel_weight(grid: dict, vox) -> float:
    """Weight of voxel ``vox`` (global integer coordinates); 0 if unallocated."""
    b = tuple(int(v) // BLOCK for v in vox)
    cell = grid.get(b)
    if cell is None:
        return 0.0
    lx, ly, lz = (int(v) - BLOCK * bb for v, bb in zip(vox, b))
    return float(cell[1][lz, ly, lx])


def novel_leaves(grid: dict, depth, lv, cam, R_cw, t_cw, voxel_size: float = 0.01):
    """Indices into ``lv`` of the leaves that seed: Eq. 10 point in a voxel
    of weight 1, at most one (smallest y0 W + x0) per voxel."""
    W = depth.shape[1]
    idx, pts = leaf_points(depth, lv, cam, R_cw, t_cw)
    s = F32(voxel_size)
    best = {}
    for n, p in zip(idx.tolist(), pts.astype(np.float32)):
        vox = tuple(int(np.floor(c / s)) for c in p)  # float32 division
        if voxel_weight(grid, vox) != 1.0:
            continue
        key = int(lv[n][1]) * W + int(lv[n][0])
        if vox not in best or key < best[vox][0]:
            best[vox] = (key, n)
    return np.array(sorted(n for _, n in best.values()), np.int64)


def seed_tsdf(rgb, depth, grid: dict, cam, R_cw, t_cw, sh_degree: int, var_thr: float = 0.01, max_size: int = 64,
              min_size: int = 1, voxel_size: float = 0.01) -> dict:
    """Quadtree of the frame, the novelty check against the integrated grid,
    then Eq. 10 for the leaves that seed."""
    lv = _qt.leaves(np.asarray(rgb, np.float64), var_thr, max_size, min_size)
    sel = novel_leaves(grid, depth, lv, cam, R_cw, t_cw, voxel_size)
    out = _qt.seed(rgb, depth, lv[sel], cam, np.asarray(R_cw, np.float64), np.asarray(t_cw, np.float64), sh_degree)
    # the means are the float32 points whose voxels were checked (Eq. 10's
    # float64 value rounded through the float32 operations)
    idx, pts = leaf_points(depth, lv[sel], cam, R_cw, t_cw)
    assert len(idx) == len(sel)
    out["means"] = pts
    return out
