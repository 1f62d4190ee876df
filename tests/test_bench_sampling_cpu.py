"""The oracle baseline's cost model: per 16 x 16 tile, the pixels times the
Gaussians whose 3-sigma box meets the tile (counted with a 2D difference
array) equal a brute-force test of every Gaussian against every tile's pixel
centres -- the same selection the oracle's tile compositing makes."""
import numpy as np


def test_tile_elements_match_brute_force():
    import bench
    from oracle import render as R
    from synth import workloads
    w = workloads.tiny_random(seed=33, n=700)
    v = w.views[0]
    got = bench.oracle_tile_elements(w)
    import torch
    with torch.no_grad():
        pr = R.project(R.to_tensors({k: np.asarray(w.params[k], np.float64) for k in R.PARAM_NAMES}), 0, v.cam,
                       np.asarray(v.pose.R, np.float64), np.asarray(v.pose.t, np.float64))
    mu = pr["mean2d"].numpy()
    cov = pr["cov2d"].numpy()
    ext = np.stack([np.sqrt(9.009 * cov[:, 0, 0]), np.sqrt(9.009 * cov[:, 1, 1])], 1)
    tx, ty = -(-v.cam.width // 16), -(-v.cam.height // 16)
    want = []
    for k in range(tx * ty):
        pix = R.tile_pixels(v.cam, [k]) + 0.5
        lo, hi = pix.min(0), pix.max(0)
        gap = np.maximum(np.maximum(lo[None] - mu, mu - hi[None]), 0.0)
        want.append(int((gap <= ext).all(1).sum()) * len(pix))
    assert np.array_equal(got, np.array(want))
