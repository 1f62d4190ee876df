"""Per-frame seeding on the GPU (gs_quadtree_leaves, gs_seed_quadtree) against
the FP64 oracle: the same leaves (as sets; the GPU emits them in no
particular order), at full frame size the defining properties on every leaf,
and the Eq. 10 parameters of the seeded Gaussians."""
import numpy as np
import pytest
import torch

from oracle import quadtree as Q
from synth import workloads
from synth.scene import Camera, look_at
from tests._util import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    ensure_built()
    from paper_2408_12677_gb300.torch_api import Context
    c = Context(0)
    yield c
    c.close()


def _gpu_leaves(ctx, rgb, thr, max_size=64, min_size=1):
    from paper_2408_12677_gb300 import abi
    t = torch.as_tensor(np.ascontiguousarray(np.transpose(rgb, (2, 0, 1)), np.float32), device="cuda")
    n = abi.gs_quadtree_leaves(ctx.handle, t, thr, max_size, min_size)
    n = -n - 1 if n < 0 else n
    out = torch.zeros((max(n, 1), 4), dtype=torch.int32, device="cuda")
    assert abi.gs_quadtree_leaves(ctx.handle, t, thr, max_size, min_size, out) == n
    return out[:n].cpu().numpy().astype(np.int64)


def _image(rng, H, W):
    rgb = rng.uniform(0, 1, (H, W, 3)) * rng.uniform(0.2, 1, (H, W))[..., None]
    rgb[: H // 3, : W // 3] = 0.4  # a flat region
    yy, xx = np.mgrid[0:H, 0:W]
    rgb[H // 2:, W // 2:] = ((xx[H // 2:, W // 2:] / W)[..., None] * np.array([1.0, 0.5, 0.2]))  # a smooth ramp
    return rgb.astype(np.float32)


@pytest.mark.parametrize("H,W,thr,max_size,min_size", [(64, 96, 0.01, 64, 1), (90, 130, 0.02, 64, 2),
                                                       (70, 150, 0.005, 32, 4), (33, 47, 0.01, 16, 1)])
def test_leaves_match_oracle(ctx, H, W, thr, max_size, min_size):
    rng = np.random.default_rng(H * W + min_size)
    rgb = _image(rng, H, W)
    got = {tuple(r) for r in _gpu_leaves(ctx, rgb, thr, max_size, min_size).tolist()}
    ref = {tuple(r) for r in Q.leaves(rgb.astype(np.float64), thr, max_size, min_size).tolist()}
    assert got == ref


def test_full_frame_leaves_satisfy_the_definition(ctx):
    """1200 x 680 frame: the leaves partition the image, and on a sample of
    leaves the oracle's cell variance confirms each decision (a leaf does not
    exceed the threshold unless it is at the minimum size; its parent does)."""
    w = workloads.single_view()
    v = w.views[0]
    rgb = np.ascontiguousarray(v.target_rgb.transpose(1, 2, 0))
    H, W = rgb.shape[:2]
    lv = _gpu_leaves(ctx, rgb, 0.01, 64, 1)
    assert lv.shape[0] > 250_000
    cov = np.zeros((H, W), np.int32)
    for x0, y0, ww, hh in lv:
        cov[y0:y0 + hh, x0:x0 + ww] += 1
    assert (cov == 1).all()
    rng = np.random.default_rng(0)
    rgb64 = rgb.astype(np.float64)
    for x0, y0, ww, hh in lv[rng.choice(lv.shape[0], 1500, replace=False)]:
        size = 1 << int(np.ceil(np.log2(max(ww, hh))))  # the cell's (unclipped) side
        if x0 % size or y0 % size:
            size = max(ww, hh)
        if size > 1 and ww * hh > 1:
            assert Q.cell_variance(rgb64, x0, y0, x0 + ww, y0 + hh) <= 0.01
        if size < 64:
            px, py = x0 - x0 % (2 * size), y0 - y0 % (2 * size)
            assert Q.cell_variance(rgb64, px, py, min(px + 2 * size, W), min(py + 2 * size, H)) > 0.01


def test_seeded_parameters_match_oracle(ctx):
    from paper_2408_12677_gb300 import abi
    from paper_2408_12677_gb300.torch_api import camera_struct
    H, W = 72, 100
    cam = Camera(90.0, 85.0, 50.0, 36.0, W, H)
    pose = look_at([0.3, -0.2, 0.1], [1.5, 3.0, 0.4])
    rng = np.random.default_rng(7)
    rgb = _image(rng, H, W)
    depth = rng.uniform(0.5, 4.0, (H, W)).astype(np.float32)
    depth[:6] = 0.0
    alpha = rng.uniform(0, 1, (H, W)).astype(np.float32)
    deg, thr = 3, 0.01
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")
    cap = 4096
    out = {"means": torch.zeros((cap, 3), device="cuda"), "log_scales": torch.zeros((cap, 3), device="cuda"),
           "quats": torch.zeros((cap, 4), device="cuda"), "opacity_logits": torch.full((cap,), 9.0, device="cuda"),
           "sh": torch.zeros((cap, 16, 3), device="cuda")}
    k = abi.gs_seed_quadtree(ctx.handle, dev(np.transpose(rgb, (2, 0, 1))), dev(depth), dev(alpha), 0.5,
                             camera_struct(cam), abi.make_viewmat(pose.R, pose.t), deg, thr, 64, 1,
                             out["means"], out["log_scales"], out["quats"], out["opacity_logits"], out["sh"], cap)
    lv = Q.leaves(rgb.astype(np.float64), thr, 64, 1)
    ref = Q.seed(rgb, depth, lv, cam, pose.R.astype(np.float64), pose.t.astype(np.float64), deg, alpha=alpha)
    assert k == ref["means"].shape[0] > 100
    assert float(out["opacity_logits"][k]) == 9.0  # nothing written past the k rows
    got = {n: t[:k].cpu().numpy().astype(np.float64) for n, t in out.items()}
    og = np.lexsort(got["means"].T)
    orf = np.lexsort(ref["means"].T)
    assert np.allclose(got["means"][og], ref["means"][orf], rtol=1e-6, atol=1e-6)
    assert np.allclose(got["log_scales"][og], ref["log_scales"][orf], rtol=1e-6, atol=1e-6)
    assert np.allclose(got["sh"][og], ref["sh"][orf], rtol=1e-6, atol=1e-6)
    assert (got["quats"] == [1, 0, 0, 0]).all() and (got["opacity_logits"] == 0).all()
    # too little room: nothing beyond capacity, the count of what was needed
    small = {n: torch.zeros_like(t) for n, t in out.items()}
    r = abi.gs_seed_quadtree(ctx.handle, dev(np.transpose(rgb, (2, 0, 1))), dev(depth), dev(alpha), 0.5,
                             camera_struct(cam), abi.make_viewmat(pose.R, pose.t), deg, thr, 64, 1,
                             small["means"][:10], small["log_scales"][:10], small["quats"][:10],
                             small["opacity_logits"][:10], small["sh"][:10], 10)
    assert r == -k - 1 and float(small["means"][10:].abs().max()) == 0.0


@pytest.mark.parametrize("novelty", ["alpha", "tsdf"])
def test_streaming_with_device_seeding(ctx, novelty):
    from paper_2408_12677_gb300.streaming import StreamingOptimizer
    st = workloads.streaming(n_frames=8, width=96, height=64, f=48.0)
    opt = StreamingOptimizer(st.cam, 1, None, iters=2, n_past=2, capacity=128, rng_seed=3,
                             seeding=dict(var_thr=0.03, min_size=4), novelty=novelty)
    stats = [opt.process_frame(*st.frame(k), st.poses[k]) for k in range(4)]
    assert stats[0].n_gaussians > 100 and stats[-1].capacity >= stats[-1].n_gaussians > stats[0].n_gaussians
    again = opt.process_frame(*st.frame(3), st.poses[3])
    assert again.new_gaussians < 0.2 * stats[0].new_gaussians
    if novelty == "tsdf":  # the repeated frame's own voxels all have weight >= 2 now
        assert again.new_gaussians < 0.05 * stats[-1].n_gaussians and again.tsdf_touched > 0
    assert torch.isfinite(opt.map.model.flat).all()
