"""Flip accounting of the TSDF comparisons (Sec. III-B.1 Eq. 6-9, the novelty
check of Sec. III-B.2).

The oracle takes every integer decision of the fusion in float64; the kernels
take them in float32.  The two may disagree only where the float64 value lies
within float32 rounding of the deciding boundary.  Every disagreement is
listed with that float64 distance; one farther from its boundary than the
float32 error bound is a failure, and the count is bounded.

Error bounds (scenes within 10 m of the origin, 0.5 m <= z <= 6 m):
* world coordinates of a band sample, an Eq. 10 point or a voxel centre in
  the camera frame: at most ~10 correctly rounded float32 operations on
  values below 32 m, each off by at most ulp(32 m) / 2 = 1.9e-6 m, so about
  4e-6 m in practice; TOL_M = 2e-5 m.
* a voxel's projection fx x / z + cx: the camera-frame error above over
  z >= 0.5 m, times fx <= 600 (1 + |x / z|), about 7e-3 px; TOL_PX = 2e-2 px.
"""
from __future__ import annotations

import numpy as np

from oracle import tsdf as T

TOL_M = 2e-5
TOL_PX = 2e-2
TSDF_TOL = 1e-4


def alloc_flips(G: set, F: np.ndarray, bs: float, budget: int | None = None):
    """Blocks the GPU touched (G) against the oracle's (from the samples F in
    block units): [(kind, block, float64 distance in metres)], oracle set.
    Raises at once if more than ``budget`` blocks differ."""
    O = T.blocks_of(F)
    n = len(G ^ O)
    assert budget is None or n <= budget, f"{n} allocation flips (budget {budget}): {sorted(G ^ O)[:5]}"
    flips = [("gpu only", b, T.block_distance(F, b) * bs) for b in sorted(G - O)]
    flips += [("oracle only", b, T.block_depth(F, b) * bs) for b in sorted(O - G)]
    return flips, O


def check_alloc(G: set, F: np.ndarray, bs: float, budget: int, log: list):
    flips, O = alloc_flips(G, F, bs, budget)
    log.extend(("alloc",) + f for f in flips)
    far = [f for f in flips if not f[2] <= TOL_M]
    assert not far, f"allocation flips beyond {TOL_M} m of a block face: {far[:5]}"
    return {b for _, b, _ in flips}


def voxel_flips(gpu_blocks: dict, ref: dict, excused: set, log: list):
    """Voxels whose weight differs, or whose tsdf differs by more than
    TSDF_TOL, between the GPU grid and the oracle grid.  A difference is a
    flip if the voxel lies in a block whose touching flipped (``excused``) or
    if, over the frames that reached it, its projection came within TOL_PX
    of a pixel edge or the image border, or its sdf within TOL_M of -eps.
    Returns (flips, far, number of voxels with weight > 0)."""
    z = np.zeros((8, 8, 8))
    inf = np.full((8, 8, 8), np.inf)
    flips, far, n = [], [], 0
    for b in sorted(set(gpu_blocks) | set(ref)):
        gt, gw = (np.asarray(a, np.float64) for a in gpu_blocks.get(b, (z, z)))
        cell = ref.get(b)
        rt, rw, mpx, msdf = (cell[0], cell[1], cell[2], cell[3]) if cell is not None else (z, z, inf, inf)
        n += int((rw > 0).sum())
        diff = (gw != rw) | ((rw > 0) & (np.abs(gt - rt) > TSDF_TOL)) | ((rw == 0) & (gt != 0))
        for zi, yi, xi in np.argwhere(diff).tolist():
            rec = (b, (xi, yi, zi), float(gw[zi, yi, xi]), float(rw[zi, yi, xi]), float(gt[zi, yi, xi]),
                   float(rt[zi, yi, xi]), float(mpx[zi, yi, xi]), float(msdf[zi, yi, xi]))
            near = b in excused or rec[6] <= TOL_PX or rec[7] <= TOL_M
            (flips if near else far).append(rec)
    log.extend(("voxel",) + f for f in flips)
    return flips, far, n


def check_voxels(gpu_blocks: dict, ref: dict, excused: set, log: list, rel_budget: float = 1e-5):
    flips, far, n = voxel_flips(gpu_blocks, ref, excused, log)
    assert not far, f"{len(far)} voxel mismatches away from any decision boundary: {far[:5]}"
    budget = max(2, int(rel_budget * n)) + 512 * len(excused)
    assert len(flips) <= budget, f"{len(flips)} voxel flips (budget {budget}): {flips[:5]}"
    return n


def _neighbour_voxel(p: np.ndarray, vox: np.ndarray, s: float) -> tuple:
    """The voxel across the face of ``vox`` nearest to point p."""
    f = p / s - vox
    d = np.concatenate([f, 1.0 - f])
    k = int(np.argmin(d))
    out = vox.copy()
    out[k % 3] += -1 if k < 3 else 1
    return tuple(out.tolist())


def flagged_voxels(rep: dict, voxel_size: float, excused_blocks: set) -> set:
    """Voxels whose seeding a float32 evaluation may decide differently: a
    leaf point in it lies within TOL_M of a voxel face (it and the voxel
    across that face), its fusion came near a decision boundary (pixel / sdf
    margins), or its block's touching flipped."""
    s = float(np.float32(voxel_size))
    pts, vox = rep["points"], rep["voxel"]
    flagged = set()
    for k in range(len(pts)):
        v = tuple(vox[k].tolist())
        b = tuple(int(c) // 8 for c in v)
        if rep["px_margin"][k] <= TOL_PX or rep["sdf_margin"][k] <= TOL_M or b in excused_blocks:
            flagged.add(v)
        if rep["voxel_margin"][k] <= TOL_M:
            flagged.add(v)
            flagged.add(_neighbour_voxel(pts[k], vox[k], s))
    return flagged


def check_seeds(got_means: np.ndarray, rep: dict, voxel_size: float, excused_blocks: set, log: list,
                budget: int | None = None):
    """Seeded means of the GPU (float32 rows, any order) against the oracle's
    novelty report: every oracle seed has a GPU mean within TOL_M and vice
    versa, except seeds of flagged voxels (``flagged_voxels``), at most
    ``budget`` of them (default: the number of flagged voxels, a flip being
    possible only there).  Returns (matched GPU rows, matched oracle leaves'
    report rows)."""
    from scipy.spatial import cKDTree
    s = float(np.float32(voxel_size))
    flagged = flagged_voxels(rep, voxel_size, excused_blocks)
    pts, vox = rep["points"], rep["voxel"]
    seed_rows = np.nonzero(rep["seeds"])[0]
    want = pts[seed_rows]
    want_vox = [tuple(v) for v in vox[seed_rows].tolist()]
    got = np.asarray(got_means, np.float64).reshape(-1, 3)
    gi, wi = [], []
    unmatched_got = list(range(len(got)))
    if len(want) and len(got):
        d, j = cKDTree(want).query(got)
        taken = set()
        unmatched_got = []
        for i in range(len(got)):
            if d[i] <= TOL_M and int(j[i]) not in taken:
                taken.add(int(j[i]))
                gi.append(i)
                wi.append(int(j[i]))
            else:
                unmatched_got.append(i)
    unmatched_want = sorted(set(range(len(want))) - set(wi))
    far = []
    for i in unmatched_got:
        v = tuple(np.floor(got[i] / s).astype(np.int64).tolist())
        rec = ("gpu only", got[i].tolist(), v)
        (log.append(("seed",) + rec) if v in flagged else far.append(rec))
    for k in unmatched_want:
        rec = ("oracle only", want[k].tolist(), want_vox[k])
        (log.append(("seed",) + rec) if want_vox[k] in flagged else far.append(rec))
    assert not far, f"{len(far)} seed mismatches away from any decision boundary: {far[:5]}"
    n_flips = len(unmatched_got) + len(unmatched_want)
    budget = len(flagged) if budget is None else budget
    assert n_flips <= budget, f"{n_flips} seed flips (budget {budget})"
    return np.array(gi, np.int64), seed_rows[np.array(wi, np.int64)] if wi else np.zeros(0, np.int64)


def census(log: list) -> str:
    """One line per flip: kind and float64 distance to the deciding boundary."""
    return "\n".join(repr(x) for x in log) if log else "no flips"
