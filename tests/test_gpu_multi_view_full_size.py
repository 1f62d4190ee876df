"""Full-size multi-view batch (8 views: 2 x 640x480, 4 x 1200x680 and
2 x 1752x1168, 7.97M pixels; 500,000 Gaussians seeded from the views; SH
degree 3) in one batched forward and one batched backward pass, the launch
configuration of the bench's multi-view comparison.  Per view, whole 16 x 16
tiles -- the two with the longest lists and four random ones -- are checked
against the oracle (colour, depth, alpha, flips audited by decision
margins), and the batched backward pass of a random upstream on those
pixels against the oracle's gradient summed over the views, with each
view's pose gradient."""
import os

import numpy as np
import pytest
import torch

from oracle import render as R
from synth import workloads
from tests._util import compare, ensure_built, oracle_params, to_gpu_model
from tests.test_gpu_batched import _batched_backward, _batched_render
from tests.test_gpu_buckets import check_visit_order
from tests.test_gpu_grad import NAMES, check_grad_arrays

pytestmark = pytest.mark.gpu

TILE = 16


@pytest.fixture(scope="module")
def setup():
    ensure_built()
    from paper_2408_12677_gb300.torch_api import Context
    w = workloads.multi_view(workers=min(8, os.cpu_count() or 1))
    c = Context(0)
    yield w, c
    c.close()


def _tile_lengths(ctx, n_tiles):
    from paper_2408_12677_gb300 import abi
    r = torch.empty((n_tiles, 2), dtype=torch.int32, device="cuda")
    abi.gs_get_tile_ranges(ctx.handle, r)
    torch.cuda.synchronize()
    r = r.cpu().numpy().view(np.uint32).astype(np.int64)
    return r[:, 1] - r[:, 0]


def test_multi_view_whole_tiles_forward_and_backward(setup):
    w, ctx = setup
    assert len(w.views) == 8 and w.n == 500_000
    model = to_gpu_model(w.params)
    imgs = _batched_render(ctx, model, w.views)
    grid = [(-(-v.cam.width // TILE), -(-v.cam.height // TILE)) for v in w.views]
    base = np.concatenate([[0], np.cumsum([tx * ty for tx, ty in grid])])
    lens = _tile_lengths(ctx, int(base[-1]))
    check_visit_order(ctx, int(base[-1]))
    P = oracle_params(w.params)
    rng = np.random.default_rng(11)
    wc, wd, wa, sel = [], [], [], []
    for v, view in enumerate(w.views):
        cam = view.cam
        local = lens[base[v]:base[v + 1]]
        longest = np.argsort(-local, kind="stable")[:2]
        rest = np.setdiff1d(np.arange(local.size), longest)
        tiles = np.concatenate([longest, rng.choice(rest, 4, replace=False)])
        pix, sizes = R.tile_pixels(cam, tiles, sizes=True)
        R64, t64 = view.pose.R.astype(np.float64), view.pose.t.astype(np.float64)
        o = R.render(P, 3, cam, R64, t64, pixels=pix, prefilter="bbox", chunk_px=sizes)
        m = R.decision_margins(w.params, 3, cam, R64, t64, pixels=pix, prefilter="bbox", chunk_px=sizes)
        mk = dict(margins=m["pixel"], kinds=m["pixel_kind"])
        budget = max(1, int(1e-5 * len(pix)))
        col, dep, alp = imgs[v]
        for c in range(3):
            compare(f"view {v} color{c}", col[c][pix[:, 1], pix[:, 0]], o["color"][c].detach().numpy(), 1e-4, 1e-6,
                    1e-4, budget, **mk)
        compare(f"view {v} depth", dep[pix[:, 1], pix[:, 0]], o["depth"].detach().numpy(), 1e-4, 1e-6, 1e-4,
                budget, **mk)
        compare(f"view {v} alpha", alp[pix[:, 1], pix[:, 0]], o["alpha"].detach().numpy(), 1e-4, 1e-6, 1e-4,
                budget, **mk)
        # the longest tiles' lists bound what the oracle blended there
        assert int(o["n_contrib"].max()) <= int(local.max())
        H, W = cam.height, cam.width
        c_img, d_img, a_img = (np.zeros((3, H, W), np.float32), np.zeros((H, W), np.float32),
                               np.zeros((H, W), np.float32))
        cw = rng.standard_normal((3, len(pix))).astype(np.float32)
        dw = rng.standard_normal(len(pix)).astype(np.float32)
        aw = rng.standard_normal(len(pix)).astype(np.float32)
        c_img[:, pix[:, 1], pix[:, 0]] = cw
        d_img[pix[:, 1], pix[:, 0]] = dw
        a_img[pix[:, 1], pix[:, 0]] = aw
        wc.append(c_img)
        wd.append(d_img)
        wa.append(a_img)
        sel.append((pix, sizes, cw, dw, aw, m))

    g = _batched_backward(ctx, model, w.views, wc, wd, wa)
    og, poses, margins = None, [], None
    for view, (pix, sizes, cw, dw, aw, m) in zip(w.views, sel):
        R64, t64 = view.pose.R.astype(np.float64), view.pose.t.astype(np.float64)
        gv, _ = R.weighted_pixel_gradients(w.params, 3, view.cam, R64, t64, pix, cw.astype(np.float64),
                                           dw.astype(np.float64), aw.astype(np.float64), prefilter="bbox",
                                           chunk_px=sizes)
        poses.append(gv["pose"])
        og = {k: gv[k] for k in NAMES} if og is None else {k: og[k] + gv[k] for k in NAMES}
        if margins is None:
            margins = {"gauss": m["gauss"].copy(), "gauss_kind": m["gauss_kind"].copy()}
        else:
            better = m["gauss"] < margins["gauss"]
            margins["gauss"][better] = m["gauss"][better]
            margins["gauss_kind"][better] = m["gauss_kind"][better]
    og["pose"] = torch.stack(poses)
    check_grad_arrays(g, og, margins)
