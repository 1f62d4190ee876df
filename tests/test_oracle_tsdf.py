"""Pins of the TSDF oracle (Sec. III-B.1, Eq. 6-9) and of its novelty check
(Sec. III-B.2) to geometry computed another way: exact segment-box
intersection for the allocation, closed-form planes seen through 4x4
homogeneous transforms for the integration, hand-expanded sums of Eq. 9,
and per-axis counts for the one-Gaussian-per-voxel rule."""
import math

import numpy as np
import pytest

from oracle import quadtree as Q
from oracle import tsdf as T
from synth.scene import Camera

S, EPS = 0.01, 0.08
BS = T.BLOCK * S
# the grid parameters are float32: expected values use the float32 numbers
S32, E32 = float(np.float32(S)), float(np.float32(EPS))


def _rot(axis, ang):
    a = np.asarray(axis, np.float64)
    a /= np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def _pose(seed):
    rng = np.random.default_rng(seed)
    R = _rot(rng.normal(size=3), rng.uniform(0.3, 1.2)).astype(np.float32)
    t = rng.uniform(-0.5, 0.5, 3).astype(np.float32)
    return R, t


def _T_cw(R, t):
    M = np.eye(4)
    M[:3, :3] = np.asarray(R, np.float64)
    M[:3, 3] = np.asarray(t, np.float64)
    return M


def _plane_depth(cam, R, t, n, c):
    """Camera-z depth of the world plane n.X = c at every pixel centre,
    through the camera-to-world transform inv(T_cw) (0 where not in front)."""
    Twc = np.linalg.inv(_T_cw(R, t))
    jj, ii = np.mgrid[0:cam.height, 0:cam.width]
    d = np.stack([(ii + 0.5 - cam.cx) / cam.fx, (jj + 0.5 - cam.cy) / cam.fy, np.ones_like(ii, float)], -1)
    dw = d @ Twc[:3, :3].T  # world direction of the ray point at camera depth 1
    C = Twc[:3, 3]
    z = (c - n @ C) / (dw @ n)
    return np.where(z > 0, z, 0.0).astype(np.float32)


def test_band_offsets():
    c = T.band_offsets(EPS, S)
    assert T.n_band_steps(EPS, S) == 4 and len(c) == 5
    assert c[0] == np.float32(-EPS) and c[-1] == np.float32(EPS) and c[2] == 0.0
    assert np.all(np.diff(c.astype(np.float64)) <= BS / 2 + 1e-7)
    assert T.n_band_steps(0.05, 0.01) == 3  # spacing 1/30 m <= 4 cm


def _segment_blocks(p0, p1):
    """Blocks (closed boxes) the segment p0-p1 meets, with the length of the
    parameter interval [0, 1] it spends in each (exact slab method)."""
    lo = np.floor(np.minimum(p0, p1) / BS).astype(int) - 1
    hi = np.floor(np.maximum(p0, p1) / BS).astype(int) + 1
    d = p1 - p0
    out = {}
    for bx in range(lo[0], hi[0] + 1):
        for by in range(lo[1], hi[1] + 1):
            for bz in range(lo[2], hi[2] + 1):
                b = np.array([bx, by, bz])
                t0, t1 = 0.0, 1.0
                for a in range(3):
                    lo_a, hi_a = b[a] * BS, (b[a] + 1) * BS
                    if abs(d[a]) < 1e-15:
                        if not lo_a <= p0[a] <= hi_a:
                            t0, t1 = 1.0, 0.0
                    else:
                        ta, tb = sorted(((lo_a - p0[a]) / d[a], (hi_a - p0[a]) / d[a]))
                        t0, t1 = max(t0, ta), min(t1, tb)
                if t1 >= t0:
                    out[(bx, by, bz)] = t1 - t0
    return out


def test_allocation_matches_exact_segment_intersection():
    """Every allocated block meets some pixel's band segment, and every block
    a segment crosses over more than one sample spacing is allocated."""
    cam = Camera(31.0, 29.0, 14.3, 9.6, 28, 20)
    R, t = _pose(3)
    rng = np.random.default_rng(4)
    depth = rng.uniform(0.6, 2.5, (cam.height, cam.width)).astype(np.float32)
    depth[rng.uniform(size=depth.shape) < 0.1] = 0.0
    A = T.allocate(depth, cam, R, t, S, EPS)
    Twc = np.linalg.inv(_T_cw(R, t))
    h = 2 * EPS / T.n_band_steps(EPS, S)
    met, must = set(), set()
    for j in range(cam.height):
        for i in range(cam.width):
            D = float(depth[j, i])
            if D <= 0:
                continue
            ray = np.array([(i + 0.5 - cam.cx) / cam.fx, (j + 0.5 - cam.cy) / cam.fy, 1.0])
            p0 = Twc[:3, :3] @ (ray * (D - EPS)) + Twc[:3, 3]
            p1 = Twc[:3, :3] @ (ray * (D + EPS)) + Twc[:3, 3]
            for b, frac in _segment_blocks(p0, p1).items():
                met.add(b)
                if frac * 2 * EPS > h + 1e-4:
                    must.add(b)
    assert len(A) > 200
    assert A <= met
    assert must <= A


def test_frontal_plane_closed_form():
    cam = Camera(40.0, 36.0, 17.0, 11.5, 36, 24)
    d = 1.013
    depth = np.full((cam.height, cam.width), d, np.float32)
    grid = {}
    A = T.integrate(grid, depth, cam, np.eye(3), np.zeros(3), S, EPS, 100.0)
    bz = {b[2] for b in A}
    assert bz == set(range(int(np.floor((d - EPS) / BS)), int(np.floor((d + EPS) / BS)) + 1))
    checked = 0
    for b, (ts, ws, *_) in grid.items():
        for lz in range(8):
            for ly in range(8):
                for lx in range(8):
                    g = np.array([8 * b[0] + lx, 8 * b[1] + ly, 8 * b[2] + lz])
                    p = (g + 0.5) * S32
                    u, v = cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy
                    sdf = float(np.float32(d)) - p[2]
                    if min(abs(u), abs(u - cam.width), abs(v), abs(v - cam.height)) < 1e-4 or abs(sdf + E32) < 1e-6:
                        continue
                    inside = 0 <= u < cam.width and 0 <= v < cam.height
                    want_w = 1.0 if inside and sdf >= -E32 else 0.0
                    assert ws[lz, ly, lx] == want_w
                    if want_w:
                        assert ts[lz, ly, lx] == pytest.approx(np.clip(sdf / E32, -1, 1), abs=1e-9)
                        checked += 1
    assert checked > 5000


def test_tilted_plane_general_pose():
    """A tilted world plane seen from a rotated, translated camera: each
    updated voxel carries (D(pixel) - z_c) / eps for the pixel its centre
    projects to through the 4x4 transform."""
    cam = Camera(33.0, 27.0, 15.2, 12.7, 32, 22)
    R, t = _pose(11)
    Twc = np.linalg.inv(_T_cw(R, t))
    n = np.array([0.3, -0.4, 0.87])
    n /= np.linalg.norm(n)
    c = n @ (Twc[:3, :3] @ np.array([0.1, -0.05, 1.6]) + Twc[:3, 3])
    depth = _plane_depth(cam, R, t, n, c)
    assert (depth > 0).all() and depth.std() > 0.05
    grid = {}
    T.integrate(grid, depth, cam, R, t, S, EPS, 100.0)
    Tcw = _T_cw(R, t)
    upd = skipped = 0
    for b, (ts, ws, *_) in grid.items():
        lz, ly, lx = np.meshgrid(range(8), range(8), range(8), indexing="ij")
        g = np.stack([8 * b[0] + lx, 8 * b[1] + ly, 8 * b[2] + lz], -1).reshape(-1, 3)
        pc = (np.c_[(g + 0.5) * S32, np.ones(512)] @ Tcw.T)[:, :3]
        u = cam.fx * pc[:, 0] / pc[:, 2] + cam.cx
        v = cam.fy * pc[:, 1] / pc[:, 2] + cam.cy
        for k in range(512):
            fu, fv = u[k] - np.floor(u[k]), v[k] - np.floor(v[k])
            if min(fu, 1 - fu, fv, 1 - fv) < 1e-3:
                skipped += 1
                continue
            inside = 0 <= u[k] < cam.width and 0 <= v[k] < cam.height
            sdf = float(depth[int(np.floor(v[k])), int(np.floor(u[k]))]) - pc[k, 2] if inside else -1e9
            if abs(sdf + E32) < 1e-5:
                skipped += 1
                continue
            z, y, x = np.unravel_index(k, (8, 8, 8))
            if inside and sdf >= -E32:
                assert ws[z, y, x] == 1.0
                assert ts[z, y, x] == pytest.approx(np.clip(sdf / E32, -1, 1), abs=1e-9)
                upd += 1
            else:
                assert ws[z, y, x] == 0.0
    assert upd > 3000 and skipped < 0.05 * 512 * len(grid)


def _column_voxel(cam, frames, fusion, w_max):
    """tsdf and weight of the voxel on the optical axis at z = 1.005 after
    integrating constant-depth frames (identity pose)."""
    grid = {}
    for d in frames:
        T.integrate(grid, np.full((cam.height, cam.width), d, np.float32), cam, np.eye(3), np.zeros(3), S, EPS,
                    w_max, fusion)
    g = np.floor(np.array([0.0, 0.0, 1.005]) / S).astype(int)
    b = tuple(g // 8)
    lx, ly, lz = g - 8 * np.array(b)
    return grid[b][0][lz, ly, lx], grid[b][1][lz, ly, lx]


@pytest.mark.parametrize("fusion", ["printed", "unit"])
def test_eq9_weighting(fusion):
    cam = Camera(20.0, 20.0, 8.0, 8.0, 16, 16)  # pixel (8, 8)'s corner on the optical axis
    ds = [1.02, 0.995, 1.041, 1.01]
    zc = (np.floor(1.005 / S) + 0.5) * S32  # centre of the voxel holding z = 1.005
    x = [np.clip((float(np.float32(d)) - zc) / E32, -1, 1) for d in ds]
    t3, w3 = _column_voxel(cam, ds[:3], fusion, 100.0)
    assert w3 == 3.0
    want = (2 * x[0] + 4 * x[1] + 9 * x[2]) / 15 if fusion == "printed" else (x[0] + x[1] + x[2]) / 3
    assert t3 == pytest.approx(want, abs=1e-12)
    # saturation at w_max = 2: Eq. 8 caps the weight
    t4, w4 = _column_voxel(cam, ds, fusion, 2.0)
    assert w4 == 2.0
    if fusion == "printed":  # weights (w_{k-1}, w_k) = (2, 2) from frame 3 on: plain halving
        t2 = (x[0] + 2 * x[1]) / 3
        want = ((t2 + x[2]) / 2 + x[3]) / 2
    else:
        want = (2 * x[0] + 2 * x[1] + 2 * x[2] + 3 * x[3]) / 9
    assert t4 == pytest.approx(want, abs=1e-12)
    # a constant measurement is a fixed point of either average
    tc, _ = _column_voxel(cam, [1.03] * 5, fusion, 3.0)
    assert tc == pytest.approx(np.clip((float(np.float32(1.03)) - zc) / E32, -1, 1), abs=1e-12)


def test_novelty_one_gaussian_per_voxel():
    """1 px leaves on a frontal plane: one seed per voxel the back-projected
    pixel centres fall in (counted per axis), won by the leaf with the
    smallest row-major corner; a second pass over the same frame seeds none."""
    cam = Camera(300.0, 260.0, 21.0, 14.0, 40, 28)
    d = 1.005
    rng = np.random.default_rng(5)
    rgb = rng.uniform(0, 1, (cam.height, cam.width, 3)).astype(np.float32)
    depth = np.full((cam.height, cam.width), d, np.float32)
    grid = {}
    T.integrate(grid, depth, cam, np.eye(3), np.zeros(3), S, EPS, 100.0)
    lv = Q.leaves(rgb.astype(np.float64), 0.0, 64, 1)
    assert (lv[:, 2:] == 1).all()
    sel = T.novel_leaves(grid, depth, lv, cam, np.eye(3), np.zeros(3), S)
    zf = float(np.float32(d))

    def axis(n, f, c):  # voxel index of each pixel column / row, and whether the voxel centre is in view
        vox = [int(np.floor((((k + 0.5) - c) * zf / f) / S)) for k in range(n)]
        first = {}
        for k, ix in enumerate(vox):
            first.setdefault(ix, k)
        seen = {ix: 0 <= f * ((ix + 0.5) * S) / ((100 + 0.5) * S) + c < n for ix in first}
        return {ix: k for ix, k in first.items() if seen[ix]}

    fx_ = axis(cam.width, cam.fx, cam.cx)
    fy_ = axis(cam.height, cam.fy, cam.cy)
    want = sorted(j * cam.width + i for i in fx_.values() for j in fy_.values())
    got = sorted(int(lv[n][1]) * cam.width + int(lv[n][0]) for n in sel)
    assert len(want) > 20 and got == want
    T.integrate(grid, depth, cam, np.eye(3), np.zeros(3), S, EPS, 100.0)
    assert len(T.novel_leaves(grid, depth, lv, cam, np.eye(3), np.zeros(3), S)) == 0


def test_novelty_partial_overlap():
    """Frame 1 sees the left half only; frame 2 (same pose) sees everything:
    frame 2 seeds only leaves whose voxel frame 1 did not update."""
    cam = Camera(60.0, 60.0, 24.0, 16.0, 48, 32)
    R, t = _pose(8)
    Twc = np.linalg.inv(_T_cw(R, t))
    n = np.array([0.1, 0.2, 0.97])
    n /= np.linalg.norm(n)
    depth = _plane_depth(cam, R, t, n, n @ (Twc[:3, :3] @ np.array([0.0, 0.0, 1.2]) + Twc[:3, 3]))
    half = depth.copy()
    half[:, cam.width // 2:] = 0.0
    rng = np.random.default_rng(9)
    rgb = rng.uniform(0, 1, (cam.height, cam.width, 3)).astype(np.float32)
    lv = Q.leaves(rgb.astype(np.float64), 0.0, 64, 2)
    grid = {}
    T.integrate(grid, half, cam, R, t, S, EPS, 100.0)
    first = T.novel_leaves(grid, half, lv, cam, R, t, S)
    snapshot = {b: c[1].copy() for b, c in grid.items()}
    T.integrate(grid, depth, cam, R, t, S, EPS, 100.0)
    second = T.novel_leaves(grid, depth, lv, cam, R, t, S)
    assert len(first) > 30 and len(second) > 30
    idx, pts = T.leaf_points(depth, lv, cam, R, t)
    where = dict(zip(idx.tolist(), pts))
    for k in second:
        vox = np.floor(where[int(k)] / np.float32(S)).astype(int)
        b = tuple(vox // 8)
        lx, ly, lz = vox - 8 * np.array(b)
        assert b not in snapshot or snapshot[b][lz, ly, lx] == 0.0
    assert np.median(lv[second, 0]) > cam.width // 2 - 2


def test_seed_tsdf_parameters():
    """The seeded Gaussians are Eq. 10 of exactly the novel leaves."""
    cam = Camera(70.0, 66.0, 20.0, 15.0, 40, 30)
    R, t = _pose(12)
    Twc = np.linalg.inv(_T_cw(R, t))
    n = np.array([-0.2, 0.1, 0.97])
    n /= np.linalg.norm(n)
    depth = _plane_depth(cam, R, t, n, n @ (Twc[:3, :3] @ np.array([0.0, 0.0, 1.4]) + Twc[:3, 3]))
    rng = np.random.default_rng(2)
    rgb = rng.uniform(0, 1, (cam.height, cam.width, 3)).astype(np.float32)
    grid = {}
    T.integrate(grid, depth, cam, R, t, S, EPS, 100.0)
    out = T.seed_tsdf(rgb, depth, grid, cam, R, t, 1, 0.001, 8, 1, S)
    lv = Q.leaves(rgb.astype(np.float64), 0.001, 8, 1)
    sel = T.novel_leaves(grid, depth, lv, cam, R, t, S)
    assert out["means"].shape[0] == len(sel) > 10
    idx, pts = T.leaf_points(depth, lv, cam, R, t)
    where = dict(zip(idx.tolist(), pts))
    assert np.allclose(out["means"], np.array([where[int(k)] for k in sel]), atol=1e-12)
    vox = {tuple(np.floor(m / np.float32(S)).astype(int)) for m in out["means"]}
    assert len(vox) == len(sel)
