"""The oracle baseline's pixel sample keeps every Gaussian that can reach a
sampled pixel: the summed-area-table selection equals a brute-force test of
each Gaussian's box against each sampled pixel centre."""
import numpy as np


def test_near_selection_matches_brute_force():
    import bench
    rng = np.random.default_rng(0)
    W, H = 37, 23
    n = 4000
    mu = np.stack([rng.uniform(-10, W + 10, n), rng.uniform(-10, H + 10, n)], 1)
    rad = rng.uniform(0.0, 6.0, n)
    rad[:50] = 0.0  # degenerate boxes
    mu[50:60] = np.array([[3.5, 4.5]]) + rng.integers(-2, 3, (10, 2))  # centres exactly on pixel centres
    for k in (1, 7, 200):
        pix = np.stack([rng.integers(0, W, k), rng.integers(0, H, k)], 1)
        got = bench.gaussians_near_pixels(mu, rad, pix, W, H)
        c = pix.astype(np.float64) + 0.5
        want = ((np.abs(mu[:, None, 0] - c[None, :, 0]) <= rad[:, None]) &
                (np.abs(mu[:, None, 1] - c[None, :, 1]) <= rad[:, None])).any(1)
        assert np.array_equal(got, want)
