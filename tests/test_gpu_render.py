"""Forward pass on the GPU vs the FP64 oracle: projected quantities and
rendered colour / depth / alpha images, over several tile shapes, SH degrees,
ragged image sizes and degenerate scenes.

Image tolerance: per channel ||g - o|| / ||o|| <= 1e-4 and element-wise
|g - o| <= 1e-4 |o| + 1e-6, except for a budget of max(1, 1e-5 x pixels)
pixels where a float32 decision (q <= 9, alpha >= 1/255, T (1 - alpha) <
1e-4, the 0.99 clamp) falls the other way than in float64 ("flips").  Every
pixel beyond the tolerance must lie within 1e-4 (relative) of one of those
thresholds in the oracle's float64 evaluation (``R.decision_margins``); it is
reported with the threshold and its distance."""
import numpy as np
import pytest
import torch

from oracle import render as R
from synth import workloads
from synth.scene import Camera, Pose, look_at
from tests._util import compare, ensure_built, gpu_render, oracle_params, to_gpu_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    ensure_built()
    from paper_2408_12677_gb300.torch_api import Context
    c = Context(0)
    yield c
    c.close()


def _flip_budget(npx):
    return max(1, int(1e-5 * npx))


def _check_images(w_params, deg, cam, pose, ctx, report=None, **cfg):
    model = to_gpu_model(w_params)
    col, dep, alp = gpu_render(ctx, model, cam, pose, **cfg)
    bg = cfg.get("bg", (0.0, 0.0, 0.0))
    rcfg = R.RasterCfg(bg=tuple(bg))
    R64, t64 = pose.R.astype(np.float64), pose.t.astype(np.float64)
    o = R.render(oracle_params(w_params), deg, cam, R64, t64, rcfg, prefilter=True)
    m = R.decision_margins(w_params, deg, cam, R64, t64, rcfg)
    npx = cam.width * cam.height
    mk = dict(margins=m["pixel"], kinds=m["pixel_kind"])
    for c in range(3):
        compare(f"color{c}", col[c], o["color"][c].detach().numpy(), 1e-4, 1e-6, 1e-4, _flip_budget(npx), report,
                **mk)
    compare("depth", dep, o["depth"].detach().numpy(), 1e-4, 1e-6, 1e-4, _flip_budget(npx), report, **mk)
    compare("alpha", alp, o["alpha"].detach().numpy(), 1e-4, 1e-6, 1e-4, _flip_budget(npx), report, **mk)
    return model, o


@pytest.mark.parametrize("tile", [(16, 16), (8, 32), (32, 8)])
def test_tiny_random_scene(ctx, tile):
    w = workloads.tiny_random()
    v = w.views[0]
    _check_images(w.params, 0, v.cam, v.pose, ctx, tile_w=tile[0], tile_h=tile[1])


def test_sh_degree3_ragged_image_posed_camera(ctx):
    cam = Camera(90.0, 85.0, 50.0, 35.0, 100, 70)  # 7 x 5 tiles of 16, ragged tail
    pose = look_at([0.2, -0.3, 0.1], [1.0, 3.0, 0.4])
    rng = np.random.default_rng(77)
    P = workloads.random_gaussians(rng, 1500, cam, pose, 3, sh_rest_std=0.15)
    _check_images(P, 3, cam, pose, ctx)


@pytest.mark.parametrize("deg", [1, 2])
def test_intermediate_sh_degrees(ctx, deg):
    cam = Camera(60.0, 60.0, 32.0, 24.0, 64, 48)
    pose = Pose(np.eye(3, dtype=np.float32), np.zeros(3, np.float32))
    P = workloads.random_gaussians(np.random.default_rng(deg), 400, cam, pose, deg, sh_rest_std=0.2)
    _check_images(P, deg, cam, pose, ctx)


def test_background_and_projection(ctx):
    w = workloads.tiny_random(seed=1010, n=300)
    v = w.views[0]
    model, o = _check_images(w.params, 0, v.cam, v.pose, ctx, bg=(0.2, 0.5, 0.9))
    from paper_2408_12677_gb300 import abi
    n = w.n
    m2 = torch.empty((n, 2), device="cuda")
    cov = torch.empty((n, 3), device="cuda")
    dep = torch.empty(n, device="cuda")
    rgb = torch.empty((n, 3), device="cuda")
    op = torch.empty(n, device="cuda")
    tiles = torch.empty(n, dtype=torch.int32, device="cuda")
    abi.gs_get_projection(ctx.handle, m2, cov, dep, rgb, op, tiles)
    torch.cuda.synchronize()
    pr = o["proj"]
    idx = pr["idx"].numpy()
    assert (tiles.cpu().numpy()[np.setdiff1d(np.arange(n), idx)] == 0).all()
    compare("mean2d", m2.cpu().numpy()[idx], pr["mean2d"].detach().numpy(), 1e-6, 1e-5, 1e-6)
    c = pr["cov2d"].detach().numpy()
    compare("cov2d", cov.cpu().numpy()[idx], np.stack([c[:, 0, 0], c[:, 0, 1], c[:, 1, 1]], 1), 1e-4, 1e-6, 1e-5)
    compare("depth", dep.cpu().numpy()[idx], pr["depth"].detach().numpy(), 1e-6, 0, 1e-7)
    compare("rgb", rgb.cpu().numpy()[idx], pr["rgb"].detach().numpy(), 1e-5, 1e-6, 1e-6)
    compare("opacity", op.cpu().numpy()[idx], pr["opacity"].detach().numpy(), 1e-5, 1e-7, 1e-6)


def test_degenerate_scenes(ctx):
    cam = Camera(60.0, 60.0, 32.0, 24.0, 64, 48)
    pose = Pose(np.eye(3, dtype=np.float32), np.zeros(3, np.float32))
    empty = {"means": np.zeros((0, 3), np.float32), "log_scales": np.zeros((0, 3), np.float32),
             "quats": np.zeros((0, 4), np.float32), "opacity_logits": np.zeros(0, np.float32),
             "sh": np.zeros((0, 1, 3), np.float32), "sh_degree": 0}
    col, dep, alp = gpu_render(ctx, to_gpu_model(empty), cam, pose, bg=(0.1, 0.2, 0.3))
    assert np.allclose(col[0], 0.1) and np.allclose(col[2], 0.3) and not dep.any() and not alp.any()
    # everything behind the camera or inside the near plane
    w = workloads.tiny_random(seed=3, n=100)
    P = dict(w.params)
    P["means"] = P["means"].copy()
    P["means"][:, 2] = np.where(np.arange(100) % 2 == 0, -P["means"][:, 2], 0.1)
    col, dep, alp = gpu_render(ctx, to_gpu_model(P), cam, pose)
    assert not col.any() and not alp.any()
    # a single large opaque Gaussian in front: alpha clamps at 0.99 over the centre
    one = {"means": np.array([[0.0, 0.0, 1.0]], np.float32), "log_scales": np.full((1, 3), np.log(2.0), np.float32),
           "quats": np.array([[1.0, 0, 0, 0]], np.float32), "opacity_logits": np.array([9.0], np.float32),
           "sh": np.full((1, 1, 3), 1.0, np.float32), "sh_degree": 0}
    _check_images(one, 0, cam, pose, ctx)
    # extremely elongated splats (needle-like), anisotropic large Gaussians
    rng = np.random.default_rng(9)
    P = workloads.random_gaussians(rng, 200, cam, pose, 0, log_scale_range=(-6.0, 0.0))
    P["opacity_logits"] = np.full(200, 2.0, np.float32)
    _check_images(P, 0, cam, pose, ctx)
