"""Full-size single view (1200x680, about 300k quadtree-seeded Gaussians, SH
degree 3) in the launch configuration the bench times: whole 16 x 16 tiles
(the 16 with the longest lists and 48 random ones) vs the oracle for every
output and the backward pass on their pixels, sampled pixels, a
sparse-upstream gradient, the blended-pair counter against the oracle's on a
crop camera, and invariants of a whole fwd + loss + bwd + Adam iteration.
The scale-stress configuration (1752x1168, 1M Gaussians, 20% large ones,
about 1.1e9 (tile, Gaussian) pairs, every tile list longer than the per-tile
sort holds, so binning takes the radix path) is checked on 64 x 64 crops."""
import numpy as np
import pytest
import torch

from oracle import render as R
from synth import workloads
from synth.scene import Camera
from tests._util import compare, ensure_built, gpu_backward, gpu_render, oracle_params, to_gpu_model

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


def _tile_lengths(ctx, n_tiles):
    from paper_2408_12677_gb300 import abi
    r = torch.empty((n_tiles, 2), dtype=torch.int32, device="cuda")
    abi.gs_get_tile_ranges(ctx.handle, r)
    torch.cuda.synchronize()
    r = r.cpu().numpy().view(np.uint32).astype(np.int64)
    return r[:, 1] - r[:, 0]


def _check_tiles(ctx, model, w, deg, cam, pose, col, dep, alp, tiles, with_grad, report=None):
    """Every output on the pixels of ``tiles`` vs the oracle (bounding-box
    selection per tile), flips audited by decision margins; with_grad: the
    backward pass of a random upstream on those pixels."""
    from tests.test_gpu_grad import check_grad_arrays
    pix, sizes = R.tile_pixels(cam, tiles, sizes=True)
    R64, t64 = pose.R.astype(np.float64), pose.t.astype(np.float64)
    o = R.render(oracle_params(w.params), deg, cam, R64, t64, pixels=pix, prefilter="bbox", chunk_px=sizes)
    m = R.decision_margins(w.params, deg, cam, R64, t64, pixels=pix, prefilter="bbox", chunk_px=sizes)
    mk = dict(margins=m["pixel"], kinds=m["pixel_kind"])
    budget = max(1, int(1e-5 * len(pix)))
    for c in range(3):
        compare(f"color{c}", col[c][pix[:, 1], pix[:, 0]], o["color"][c].detach().numpy(), 1e-4, 1e-6, 1e-4,
                budget, report, **mk)
    compare("depth", dep[pix[:, 1], pix[:, 0]], o["depth"].detach().numpy(), 1e-4, 1e-6, 1e-4, budget, report, **mk)
    compare("alpha", alp[pix[:, 1], pix[:, 0]], o["alpha"].detach().numpy(), 1e-4, 1e-6, 1e-4, budget, report, **mk)
    if not with_grad:
        return o
    rng = np.random.default_rng(len(tiles))
    H, W = cam.height, cam.width
    wc = rng.standard_normal((3, len(pix))).astype(np.float32)
    wd = rng.standard_normal(len(pix)).astype(np.float32)
    wa = rng.standard_normal(len(pix)).astype(np.float32)
    wc_img, wd_img, wa_img = np.zeros((3, H, W), np.float32), np.zeros((H, W), np.float32), np.zeros((H, W), np.float32)
    wc_img[:, pix[:, 1], pix[:, 0]] = wc
    wd_img[pix[:, 1], pix[:, 0]] = wd
    wa_img[pix[:, 1], pix[:, 0]] = wa
    g = gpu_backward(ctx, model, cam, pose, wc_img, wd_img, wa_img)
    og, _ = R.weighted_pixel_gradients(w.params, deg, cam, R64, t64, pix, wc.astype(np.float64),
                                       wd.astype(np.float64), wa.astype(np.float64), prefilter="bbox",
                                       chunk_px=sizes)
    check_grad_arrays(g, og, m, report=report)
    return o


def test_whole_tiles_including_the_longest_lists(setup):
    w, ctx = setup
    v = w.views[0]
    model = to_gpu_model(w.params)
    col, dep, alp = gpu_render(ctx, model, v.cam, v.pose)
    tx, ty = -(-v.cam.width // 16), -(-v.cam.height // 16)
    lens = _tile_lengths(ctx, tx * ty)
    assert lens.sum() > w.n
    longest = np.argsort(-lens, kind="stable")[:16]
    rest = np.setdiff1d(np.arange(tx * ty), longest)
    tiles = np.concatenate([longest, np.random.default_rng(3).choice(rest, 48, replace=False)])
    o = _check_tiles(ctx, model, w, 3, v.cam, v.pose, col, dep, alp, tiles, with_grad=True)
    # the tiles' list lengths bound the Gaussians the oracle blended there
    assert int(o["n_contrib"].max()) <= int(lens.max())


def _crop_camera(cam, x0, y0, size=64):
    """The camera of the size x size window at (x0, y0): the same pixel rays."""
    return Camera(cam.fx, cam.fy, cam.cx - x0, cam.cy - y0, size, size)


def _eval_counter(ctx, model, cam, pose):
    from paper_2408_12677_gb300 import abi
    abi.gs_set_eval_counting(ctx.handle, True)
    gpu_render(ctx, model, cam, pose)
    n = ctx.stats()["evals_blended"]
    abi.gs_set_eval_counting(ctx.handle, False)
    return n


def test_eval_counter_matches_oracle_on_crop_camera(setup):
    """The blended-pair counter (the numerator of the Gaussian-pixel evals/s
    metric) equals the oracle's count of blended pairs, n_contrib summed over
    the pixels of a 64 x 64 crop camera, up to the pixels within float32
    rounding of a threshold."""
    w, ctx = setup
    v = w.views[0]
    cam = _crop_camera(v.cam, 560, 300)
    got = _eval_counter(ctx, to_gpu_model(w.params), cam, v.pose)
    pix, sizes = R.tile_pixels(cam, range(16), sizes=True)
    R64, t64 = v.pose.R.astype(np.float64), v.pose.t.astype(np.float64)
    o = R.render(oracle_params(w.params), 3, cam, R64, t64, pixels=pix, prefilter="bbox", chunk_px=sizes)
    m = R.decision_margins(w.params, 3, cam, R64, t64, pixels=pix, prefilter="bbox", chunk_px=sizes)
    want = R.gaussian_pixel_evals(o)
    near = int((m["pixel"] <= 1e-4).sum())
    assert want > 50_000 and abs(got - want) <= near, (got, want, near)
