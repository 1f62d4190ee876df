"""Pins for the oracle's per-frame seeding (Sec. III-B.2, Eq. 10): the
contrast quadtree against closed cases and invariants, and the
back-projection of leaf centres against the camera model."""
import numpy as np
import pytest

from oracle import quadtree as Q
from synth import quadtree as synth_quadtree
from synth.scene import Camera, look_at


def _covers_exactly_once(lv, W, H):
    cov = np.zeros((H, W), np.int32)
    for x0, y0, w, h in lv:
        cov[y0:y0 + h, x0:x0 + w] += 1
    return bool((cov == 1).all())


def test_constant_image_gives_the_clipped_root_grid():
    rgb = np.full((150, 200, 3), 0.3)
    lv = Q.leaves(rgb)
    assert lv.shape[0] == 4 * 3  # ceil(200 / 64) x ceil(150 / 64)
    assert set(map(tuple, lv.tolist())) >= {(192, 128, 8, 22), (0, 0, 64, 64)}
    assert _covers_exactly_once(lv, 200, 150)


def test_one_pixel_checkerboard_splits_to_single_pixels():
    yy, xx = np.mgrid[0:40, 0:48]
    rgb = np.repeat(((xx + yy) % 2).astype(np.float64)[..., None], 3, 2)
    lv = Q.leaves(rgb)
    assert lv.shape[0] == 40 * 48 and (lv[:, 2] == 1).all() and (lv[:, 3] == 1).all()


def test_threshold_is_strict_on_the_variance():
    # a 64 x 64 cell, left half 0, right half s: every channel has variance s^2 / 4
    s = 0.3
    rgb = np.zeros((64, 64, 3))
    rgb[:, 32:] = s
    var = s * s / 4
    assert Q.leaves(rgb, var_thr=var * (1 + 1e-9)).shape[0] == 1
    assert Q.leaves(rgb, var_thr=var * (1 - 1e-9)).shape[0] == 4  # halves are constant: no further split


def test_min_size_and_partition_on_random_images():
    rng = np.random.default_rng(5)
    rgb = rng.uniform(0, 1, (70, 100, 3))
    rgb[:30, :40] = 0.5  # a flat region stays coarse
    for mn in (1, 2, 4):
        lv = Q.leaves(rgb, var_thr=0.02, min_size=mn)
        assert _covers_exactly_once(lv, 100, 70)
        assert (np.minimum(lv[:, 2], lv[:, 3]) >= 1).all()
        full = (lv[:, 0] + mn <= 100) & (lv[:, 1] + mn <= 70)
        assert (lv[full][:, 2] >= mn).all() and (lv[full][:, 3] >= mn).all()
        assert (lv[:, 2] <= 64).all()


def test_matches_the_integral_image_generator():
    # an independent implementation of the same rule (integral images, level by level)
    rng = np.random.default_rng(9)
    for shape, thr, mn in (((68, 120, 3), 0.01, 1), ((100, 90, 3), 0.03, 2)):
        rgb = rng.uniform(0, 1, shape) * rng.uniform(0, 1, shape[:2])[..., None]
        a = {tuple(r) for r in Q.leaves(rgb, thr, 64, mn).tolist()}
        b = {tuple(r) for r in synth_quadtree.quadtree_leaves(rgb.astype(np.float32).astype(np.float64), thr, 64,
                                                               mn).tolist()}
        assert a == b


def test_back_projection_lands_on_the_leaf_centre_ray():
    cam = Camera(300.0, 280.0, 64.0, 48.0, 128, 96)
    pose = look_at([0.3, -0.2, 0.1], [1.5, 3.0, 0.4])
    rng = np.random.default_rng(2)
    rgb = rng.uniform(0, 1, (96, 128, 3))
    depth = rng.uniform(0.5, 4.0, (96, 128))
    depth[:10] = 0.0  # invalid rows seed nothing
    alpha = rng.uniform(0, 1, (96, 128))
    lv = Q.leaves(rgb, 0.02, 64, 2)
    u, _, vt = np.linalg.svd(pose.R.astype(np.float64))  # an exactly orthonormal rotation in float64
    R, t = u @ vt, pose.t.astype(np.float64)
    P = Q.seed(rgb, depth, lv, cam, R, t, 3, alpha=alpha, alpha_thr=0.5)
    kept = []
    for x0, y0, w, h in lv:
        ux, uy = x0 + w / 2.0, y0 + h / 2.0
        pi, pj = min(int(ux), 127), min(int(uy), 95)
        if depth[pj, pi] > 0 and alpha[pj, pi] < 0.5:
            kept.append((ux, uy, depth[pj, pi], rgb[pj, pi], np.hypot(w, h)))
    assert P["means"].shape[0] == len(kept) > 50
    for (ux, uy, z, c, diag), m, ls, sh in zip(kept, P["means"], P["log_scales"], P["sh"]):
        pc = R @ m + t
        assert abs(pc[2] - z) < 1e-12
        assert abs(cam.fx * pc[0] / pc[2] + cam.cx - ux) < 1e-9 and abs(cam.fy * pc[1] / pc[2] + cam.cy - uy) < 1e-9
        assert np.allclose(np.exp(ls), 0.5 * diag * z / cam.fx, rtol=1e-12)
        assert np.allclose(0.5 + Q.Y00 * sh[0], c, atol=1e-12) and not sh[1:].any()
    assert (P["quats"] == [1, 0, 0, 0]).all() and (P["opacity_logits"] == 0).all()
