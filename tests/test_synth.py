"""Pins for the seeded input generators (quadtree seeding, Sec. III-B.2)."""
import json
import math
import os

import numpy as np
import torch

from oracle import sh as osh
from synth import quadtree, workloads
from synth.scene import Camera, look_at

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_init_constants.json")


def _cover(leaves, H, W):
    c = np.zeros((H, W), int)
    for x0, y0, w, h in leaves:
        c[y0:y0 + h, x0:x0 + w] += 1
    return c


def test_constant_image_keeps_root_cells():
    img = np.full((100, 150, 3), 0.3, np.float32)
    L = quadtree.quadtree_leaves(img)
    assert L.shape[0] == math.ceil(100 / 64) * math.ceil(150 / 64)
    assert (_cover(L, 100, 150) == 1).all()


def test_one_pixel_checkerboard_splits_to_single_pixels():
    jj, ii = np.mgrid[0:40, 0:70]
    img = np.repeat(((ii + jj) % 2).astype(np.float32)[..., None], 3, 2)
    L = quadtree.quadtree_leaves(img)
    assert (L[:, 2] == 1).all() and (L[:, 3] == 1).all() and L.shape[0] == 40 * 70


def test_leaves_partition_image(rng):
    img = rng.uniform(0, 1, (90, 130, 3)).astype(np.float32)
    img[:, :60] = 0.5
    L = quadtree.quadtree_leaves(img)
    assert (_cover(L, 90, 130) == 1).all()
    # a 64x64 root cell whose variance is just under / just over the threshold
    a = np.zeros((64, 64, 3), np.float32)
    a[:, :32] = 0.1
    a[:, 32:] = 0.1 + 2 * 0.0995  # variance 0.0995^2 < 0.01 -> leaf
    assert quadtree.quadtree_leaves(a).shape[0] == 1
    a[:, 32:] = 0.1 + 2 * 0.1005
    assert quadtree.quadtree_leaves(a).shape[0] == 4


def test_seeded_gaussians_follow_paper_init():
    """R = I, S = d I with d the back-projected half diagonal, alpha = 0.5 and
    decoded DC colour = pixel colour (Sec. III-B.2); constants from the golden
    fixture that cites the paper."""
    g = json.load(open(GOLDEN))
    cam = Camera(100.0, 100.0, 40.0, 30.0, 80, 60)
    pose = look_at([1.0, 1.0, 1.0], [4.0, 2.0, 1.2])
    rng = np.random.default_rng(3)
    rgb = rng.uniform(0, 1, (60, 80, 3)).astype(np.float32)
    depth = rng.uniform(1.0, 3.0, (60, 80)).astype(np.float32)
    P = quadtree.seed_gaussians(rgb, depth, cam, pose, 3, var_thr=g["quadtree_threshold"] ** 2)
    assert np.allclose(1 / (1 + np.exp(-P["opacity_logits"])), g["init_opacity"])
    assert (P["quats"] == np.array(g["init_rotation_quaternion"], np.float32)).all()
    assert np.allclose(P["log_scales"][:, 0], P["log_scales"][:, 1])
    L = quadtree.quadtree_leaves(rgb, g["quadtree_threshold"] ** 2)
    assert P["means"].shape[0] == L.shape[0]
    d = torch.tensor([[0.0, 0.0, 1.0]], dtype=torch.float64).repeat(L.shape[0], 1)
    col = osh.sh_to_rgb(torch.as_tensor(P["sh"][:, :1].astype(np.float64)), d, 0).numpy()
    cx = np.minimum(np.floor(L[:, 0] + L[:, 2] / 2).astype(int), 79)
    cy = np.minimum(np.floor(L[:, 1] + L[:, 3] / 2).astype(int), 59)
    np.testing.assert_allclose(col, rgb[cy, cx], atol=1e-6)
    # back-projection (Eq. 10): the mean projects back to the leaf centre at the leaf depth
    pc = P["means"].astype(np.float64) @ pose.R.T.astype(np.float64) + pose.t
    u = cam.fx * pc[:, 0] / pc[:, 2] + cam.cx
    np.testing.assert_allclose(u, L[:, 0] + L[:, 2] / 2, atol=2e-4)
    np.testing.assert_allclose(pc[:, 2], depth[cy, cx], rtol=1e-5)
    half_diag = 0.5 * np.hypot(L[:, 2], L[:, 3]) * depth[cy, cx] / cam.fx
    np.testing.assert_allclose(np.exp(P["log_scales"][:, 0]), half_diag, rtol=1e-5)


def test_tiny_random_recipe():
    w = workloads.tiny_random()
    assert w.n == 500 and w.views[0].target_rgb.shape == (3, 48, 64)
    pc = w.params["means"]
    z = pc[:, 2]
    assert (z >= 0.5).all() and (z <= 4.0).all()
    u = 60 * pc[:, 0] / z + 32
    assert (u >= -1e-3).all() and (u <= 64 + 1e-3).all()
    assert np.allclose(np.linalg.norm(w.params["quats"], axis=1), 1, atol=1e-6)
    w2 = workloads.tiny_random()
    assert all(np.array_equal(w.params[k], w2.params[k]) for k in ("means", "sh"))
