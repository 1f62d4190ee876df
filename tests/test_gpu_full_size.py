"""Full-size single view (1200x680, about 300k quadtree-seeded Gaussians, SH
degree 3) in the launch configuration the bench times: sampled pixels vs the
oracle, a sparse-upstream gradient vs the oracle, and invariants of a whole
fwd + loss + bwd + Adam iteration."""
import numpy as np
import pytest
import torch

from oracle import render as R
from synth import workloads
from tests._util import compare, ensure_built, gpu_backward, gpu_render, to_gpu_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    ensure_built()
    from paper_2408_12677_gb300.torch_api import Context
    w = workloads.single_view(sh_rest_std=0.05)
    c = Context(0)
    yield w, c
    c.close()


def test_sampled_pixels_match_oracle(setup):
    w, ctx = setup
    v = w.views[0]
    model = to_gpu_model(w.params)
    col, dep, alp = gpu_render(ctx, model, v.cam, v.pose)
    rng = np.random.default_rng(0)
    pix = np.stack([rng.integers(0, v.cam.width, 384), rng.integers(0, v.cam.height, 384)], 1)
    o = R.render(R.to_tensors({k: np.asarray(w.params[k], np.float64) for k in R.PARAM_NAMES}), 3, v.cam,
                 v.pose.R.astype(np.float64), v.pose.t.astype(np.float64), pixels=pix, prefilter=True)
    for c in range(3):
        compare(f"color{c}", col[c][pix[:, 1], pix[:, 0]], o["color"][c].detach().numpy(), 1e-4, 1e-6, 1e-4, 2)
    compare("depth", dep[pix[:, 1], pix[:, 0]], o["depth"].detach().numpy(), 1e-4, 1e-6, 1e-4, 2)
    compare("alpha", alp[pix[:, 1], pix[:, 0]], o["alpha"].detach().numpy(), 1e-4, 1e-6, 1e-4, 2)
    assert np.isfinite(col).all() and (alp >= 0).all() and (alp < 1).all()


def test_sparse_upstream_gradient_matches_oracle(setup):
    w, ctx = setup
    v = w.views[0]
    H, W = v.cam.height, v.cam.width
    model = to_gpu_model(w.params)
    gpu_render(ctx, model, v.cam, v.pose)
    rng = np.random.default_rng(1)
    pix = np.unique(np.stack([rng.integers(0, W, 200), rng.integers(0, H, 200)], 1), axis=0)
    wc_img = np.zeros((3, H, W), np.float32)
    wd_img = np.zeros((H, W), np.float32)
    wc = rng.standard_normal((3, len(pix))).astype(np.float32)
    wd = rng.standard_normal(len(pix)).astype(np.float32)
    wc_img[:, pix[:, 1], pix[:, 0]] = wc
    wd_img[pix[:, 1], pix[:, 0]] = wd
    g = gpu_backward(ctx, model, v.cam, v.pose, wc_img, wd_img, None)
    og, _ = R.weighted_pixel_gradients(w.params, 3, v.cam, v.pose.R.astype(np.float64), v.pose.t.astype(np.float64),
                                       pix, wc.astype(np.float64), wd.astype(np.float64), None, prefilter=True)
    from tests.test_gpu_grad import check_grad_arrays
    check_grad_arrays(g, og, R.decision_margins(w.params, 3, v.cam, v.pose.R.astype(np.float64),
                                                v.pose.t.astype(np.float64), pixels=pix))


def test_training_iterations_reduce_loss(setup):
    w, ctx = setup
    v = w.views[0]
    from paper_2408_12677_gb300.torch_api import Trainer
    model = to_gpu_model(w.params)
    tr = Trainer(model, v.cam, v.pose.R, v.pose.t, ctx=ctx)
    trgb = torch.as_tensor(v.target_rgb, device="cuda")
    tdep = torch.as_tensor(v.target_depth, device="cuda")
    losses = []
    for _ in range(10):
        losses.append(float(tr.step(trgb, tdep)))
    assert all(np.isfinite(losses)) and losses[-1] < losses[0]
    assert torch.isfinite(model.flat).all()
    st = ctx.stats()
    assert st["n_pairs"] > w.n and st["kernel_launches"] > 0
