"""The scale-stress configuration at full size: 1752x1168 (fx 1200), 1M
quadtree-seeded Gaussians of which 20% are large (log-scale U[-1, 0],
opacity logit +2), SH degree 3.  About 1.1e9 (tile, Gaussian) pairs and every
16 x 16 tile list longer than the per-tile sort holds, so the binning takes
the radix path (depth sort over the 1M items, duplication, pair sort by
tile).  The frame is rendered in the launch configuration the bench times;
64 x 64 crops (16 whole tiles, one of them the tile with the longest list)
are compared with the FP64 oracle on every output, the backward pass on the
longest tile's pixels, and the blended-pair counter on a crop camera."""
import numpy as np
import pytest
import torch

from oracle import render as R
from synth import workloads
from tests._util import ensure_built, gpu_render, oracle_params, to_gpu_model
from tests.test_gpu_full_size import _check_tiles, _crop_camera, _eval_counter, _tile_lengths

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stress():
    ensure_built()
    from paper_2408_12677_gb300.torch_api import Context
    w = workloads.scale_stress()
    c = Context(0)
    yield w, c
    c.close()


def _crop_tiles(tx, tile, size=4):
    """The size x size tiles of the crop holding ``tile`` (aligned to the crop grid)."""
    cx, cy = (tile % tx) // size * size, (tile // tx) // size * size
    return np.array([(cy + j) * tx + cx + i for j in range(size) for i in range(size)])


def test_scale_stress_crops_on_the_radix_path(stress):
    from paper_2408_12677_gb300 import abi
    w, ctx = stress
    v = w.views[0]
    model = to_gpu_model(w.params)
    abi.gs_set_profiling(ctx.handle, True)
    col, dep, alp = gpu_render(ctx, model, v.cam, v.pose)
    stages = abi.gs_profile_read(ctx.handle)
    abi.gs_set_profiling(ctx.handle, False)
    assert stages["depth_sort"][1] > 0  # the radix path ran
    st = ctx.stats()
    tx, ty = -(-v.cam.width // 16), -(-v.cam.height // 16)
    lens = _tile_lengths(ctx, tx * ty)
    assert st["n_pairs"] == lens.sum() > 500_000_000 and lens.min() > 4096
    assert np.isfinite(col).all() and (alp >= 0).all() and (alp < 1).all()
    longest = int(np.argmax(lens))
    tiles = _crop_tiles(tx, longest)
    tiles = tiles[tiles < tx * ty]
    _check_tiles(ctx, model, w, 3, v.cam, v.pose, col, dep, alp, tiles, with_grad=False)
    _check_tiles(ctx, model, w, 3, v.cam, v.pose, col, dep, alp, np.array([longest]), with_grad=True)


def test_scale_stress_eval_counter(stress):
    w, ctx = stress
    v = w.views[0]
    cam = _crop_camera(v.cam, 832, 544)
    got = _eval_counter(ctx, to_gpu_model(w.params), cam, v.pose)
    pix, sizes = R.tile_pixels(cam, range(16), sizes=True)
    R64, t64 = v.pose.R.astype(np.float64), v.pose.t.astype(np.float64)
    o = R.render(oracle_params(w.params), 3, cam, R64, t64, pixels=pix, prefilter="bbox", chunk_px=sizes)
    m = R.decision_margins(w.params, 3, cam, R64, t64, pixels=pix, prefilter="bbox", chunk_px=sizes)
    want = R.gaussian_pixel_evals(o)
    near = int((m["pixel"] <= 1e-4).sum())
    assert want > 4096 and abs(got - want) <= near, (got, want, near)
