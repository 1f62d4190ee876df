"""The TSDF flip accounting (tests/_tsdf_flips.py) on the CPU: a float32
evaluation of the fusion in the operation order gs_tsdf_integrate and
gs_seed_tsdf document (written here as a stand-in for the kernels) agrees
with the float64 oracle up to flips within the float32 error bounds, and a
mistake planted in the oracle (a transposed rotation, a wider band, a
different voxel size) makes the accounting fail."""
import numpy as np
import pytest

from oracle import quadtree as Q
from oracle import tsdf as T
from synth import workloads
from tests import _tsdf_flips as FL

F32 = np.float32
S, EPS = 0.01, 0.08
BS = 8 * float(F32(S))


@pytest.fixture(scope="module")
def stream():
    return workloads.streaming(n_frames=40, width=96, height=64, f=60.0)


def _f32_alloc(depth, cam, R, t):
    """Band samples' blocks in float32, the documented operation order."""
    R, t = np.asarray(R, F32), np.asarray(t, F32)
    fx, fy, cx, cy = (F32(cam.fx), F32(cam.fy), F32(cam.cx), F32(cam.cy))
    bs = F32(F32(8) * F32(S))
    dep = np.asarray(depth, F32)
    jj, ii = np.nonzero(dep > F32(0))
    D = dep[jj, ii]
    xn = ((ii.astype(F32) + F32(0.5)) - cx) / fx
    yn = ((jj.astype(F32) + F32(0.5)) - cy) / fy
    e = F32(EPS)
    n = T.n_band_steps(EPS, S)
    out = set()
    for k in range(n + 1):
        z = D + F32(-e + F32(k) * (F32(2) * e / F32(n)))
        ok = z > F32(0)
        pc = (xn[ok] * z[ok], yn[ok] * z[ok], z[ok])
        d = [pc[r] - t[r] for r in range(3)]
        blk = [np.floor(((R[0, a] * d[0] + R[1, a] * d[1]) + R[2, a] * d[2]) / bs).astype(np.int64) for a in range(3)]
        out.update(zip(blk[0].tolist(), blk[1].tolist(), blk[2].tolist()))
    return out


def _f32_integrate(grid, blocks, depth, cam, R, t, w_max=100.0):
    """Eq. 6-9 with float32 decisions (pixel, update) and float32 values."""
    H, W = depth.shape
    R, t = np.asarray(R, F32), np.asarray(t, F32)
    fx, fy, cx, cy = (F32(cam.fx), F32(cam.fy), F32(cam.cx), F32(cam.cy))
    s, e = F32(S), F32(EPS)
    dep = np.asarray(depth, F32)
    lz, ly, lx = (a.ravel() for a in np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij"))
    for b in blocks:
        g = [8 * b[a] + l for a, l in enumerate((lx, ly, lz))]
        pv = [(ga.astype(F32) + F32(0.5)) * s for ga in g]
        pc = [((R[r, 0] * pv[0] + R[r, 1] * pv[1]) + R[r, 2] * pv[2]) + t[r] for r in range(3)]
        with np.errstate(divide="ignore", invalid="ignore"):
            u = fx * (pc[0] / pc[2]) + cx
            v = fy * (pc[1] / pc[2]) + cy
        ok = (pc[2] > 0) & (u >= 0) & (u < W) & (v >= 0) & (v < H)
        pi = np.where(ok, np.floor(np.where(ok, u, 0)), 0).astype(np.int64)
        pj = np.where(ok, np.floor(np.where(ok, v, 0)), 0).astype(np.int64)
        D = dep[pj, pi]
        sdf = D - pc[2]
        upd = ok & (D > 0) & (sdf >= -e)
        ts = np.clip(sdf / e, -1, 1)
        cell = grid.setdefault(tuple(b), (np.zeros((8, 8, 8), F32), np.zeros((8, 8, 8), F32)))
        zi, yi, xi = lz[upd], ly[upd], lx[upd]
        w_old = cell[1][zi, yi, xi]
        w_new = np.minimum(F32(w_max), w_old + F32(1))
        cell[0][zi, yi, xi] = (cell[0][zi, yi, xi] * w_old + ts[upd] * w_new) / (w_old + w_new)
        cell[1][zi, yi, xi] = w_new


def _f32_points(depth, lv, cam, R, t):
    H, W = depth.shape
    R, t = np.asarray(R, F32), np.asarray(t, F32)
    fx, fy, cx, cy = (F32(cam.fx), F32(cam.fy), F32(cam.cx), F32(cam.cy))
    pts = []
    for x0, y0, w, h in np.asarray(lv, np.int64):
        ux, uy = F32(x0 + w / 2.0), F32(y0 + h / 2.0)
        pi, pj = min(int(np.floor(ux)), W - 1), min(int(np.floor(uy)), H - 1)
        z = F32(depth[pj, pi])
        if not z > 0:
            continue
        q = [((ux - cx) * z) / fx - t[0], ((uy - cy) * z) / fy - t[1], z - t[2]]
        pts.append([(R[0, a] * q[0] + R[1, a] * q[1]) + R[2, a] * q[2] for a in range(3)])
    return np.array(pts, F32).reshape(-1, 3)


def _frames(stream, ks):
    for k in ks:
        rgb, depth = stream.frame(k)
        yield rgb, depth, stream.poses[k]


def test_float32_allocation_agrees_up_to_logged_flips(stream):
    log = []
    for _, depth, pose in _frames(stream, (0, 5, 11)):
        G = _f32_alloc(depth, stream.cam, pose.R, pose.t)
        F = T.allocation_samples(depth, stream.cam, pose.R, pose.t, S, EPS)
        FL.check_alloc(G, F, BS, budget=max(2, len(G) // 50), log=log)
    assert all(d <= FL.TOL_M for *_, d in log)


def test_planted_transposed_rotation_in_the_oracle_fails(stream):
    _, depth, pose = next(_frames(stream, (5,)))
    G = _f32_alloc(depth, stream.cam, pose.R, pose.t)
    F = T.allocation_samples(depth, stream.cam, np.asarray(pose.R).T, pose.t, S, EPS)
    with pytest.raises(AssertionError):
        FL.check_alloc(G, F, BS, budget=10, log=[])


def test_float32_integration_agrees_up_to_logged_flips(stream):
    g32, ref, log, excused = {}, {}, [], set()
    for _, depth, pose in _frames(stream, (0, 4, 8)):
        G = _f32_alloc(depth, stream.cam, pose.R, pose.t)
        F = T.allocation_samples(depth, stream.cam, pose.R, pose.t, S, EPS)
        excused |= FL.check_alloc(G, F, BS, budget=max(2, len(G) // 50), log=log)
        _f32_integrate(g32, sorted(G), depth, stream.cam, pose.R, pose.t)
        T.integrate_blocks(ref, sorted(T.blocks_of(F)), depth, stream.cam, pose.R, pose.t, S, EPS, 100.0)
    assert FL.check_voxels(g32, ref, excused, log) > 50_000


def test_planted_wider_band_in_the_oracle_fails(stream):
    g32, ref = {}, {}
    _, depth, pose = next(_frames(stream, (3,)))
    G = _f32_alloc(depth, stream.cam, pose.R, pose.t)
    _f32_integrate(g32, sorted(G), depth, stream.cam, pose.R, pose.t)
    T.integrate_blocks(ref, sorted(G), depth, stream.cam, pose.R, pose.t, S, 0.09, 100.0)
    with pytest.raises(AssertionError):
        FL.check_voxels(g32, ref, set(), [])


def test_float32_seed_points_agree_up_to_logged_flips(stream):
    ref, log = {}, []
    for rgb, depth, pose in _frames(stream, (0, 6)):
        T.integrate(ref, depth, stream.cam, pose.R, pose.t)
        lv = Q.leaves(np.asarray(rgb, np.float64), 0.01, 16, 1)
        rep = T.novelty(ref, depth, lv, stream.cam, pose.R, pose.t, S)
        p32 = _f32_points(depth, lv, stream.cam, pose.R, pose.t).astype(np.float64)
        assert np.abs(p32 - rep["points"]).max() <= FL.TOL_M  # the float32 error bound of an Eq. 10 point
        got = p32[rep["seeds"]]
        FL.check_seeds(got, rep, S, set(), log, budget=2)
        # planted: a seed moved to another voxel is a mismatch away from any boundary
        bad = got.copy()
        bad[0] += 3 * S
        with pytest.raises(AssertionError):
            FL.check_seeds(bad, rep, S, set(), [], budget=2)
