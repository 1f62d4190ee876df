"""Pins for the integer binning oracle: brute-force tile/box overlap with
exact rational arithmetic, Python's sorted() on (tile, depth, id), and the
range boundaries; plus edge cases."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import binning


def _brute(mean2d, extent, depth, W, H, tw, th):
    TX, TY = -(-W // tw), -(-H // th)
    rows = []
    for g in range(len(mean2d)):
        mx, my = (Fraction(float(v)) for v in mean2d[g])
        ex, ey = (Fraction(float(v)) for v in extent[g])
        if ex <= 0 or ey <= 0:
            continue
        for ty in range(TY):
            for tx in range(TX):
                # closed box [m - e, m + e] meets the half-open tile [t*tw, (t+1)*tw)
                if mx - ex < (tx + 1) * tw and mx + ex >= tx * tw and my - ey < (ty + 1) * th and my + ey >= ty * th:
                    rows.append((ty * TX + tx, float(np.float32(depth[g])), g))
    return sorted(rows), TX * TY


@pytest.mark.parametrize("tw,th", [(16, 16), (8, 32), (32, 8)])
def test_matches_brute_force_on_exact_inputs(tw, th, rng):
    W, H, n = 100, 70, 60
    # quarter-pixel values: every float32 operation of the rule is exact
    mean2d = rng.integers(-40, 4 * 120, (n, 2)) / 4.0
    extent = rng.integers(0, 4 * 30, (n, 2)) / 4.0
    depth = rng.integers(1, 6, n).astype(np.float32) * 0.5  # many equal depths: tests the id tie-break
    keys, ids, ranges = binning.bin_tiles(mean2d, extent, depth, W, H, tw, th)
    rows, T = _brute(mean2d, extent, depth, W, H, tw, th)
    assert len(rows) == keys.size
    assert [r[0] for r in rows] == (keys >> np.uint64(32)).astype(np.int64).tolist()
    assert [r[2] for r in rows] == ids.tolist()
    zb = np.asarray([r[1] for r in rows], np.float32).view(np.uint32)
    assert (zb == (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)).all()
    for t in range(T):
        want = [r[2] for r in rows if r[0] == t]
        lo, hi = ranges[t]
        assert ids[lo:hi].tolist() == want
        if not want:
            assert lo == hi == 0


def test_edge_cases():
    k, i, r = binning.bin_tiles(np.zeros((0, 2)), np.zeros((0, 2)), np.zeros(0), 64, 48, 16, 16)
    assert k.size == 0 and i.size == 0 and r.shape == (12, 2) and not r.any()
    # non-participating (zero extent) and fully off-screen Gaussians emit nothing
    m = np.array([[10.0, 10.0], [-100.0, 10.0], [500.0, 500.0]])
    e = np.array([[0.0, 4.0], [5.0, 5.0], [5.0, 5.0]])
    k, i, r = binning.bin_tiles(m, e, np.ones(3), 64, 48, 16, 16)
    assert k.size == 0
    # a Gaussian covering the whole image lists every tile once, in order
    k, i, r = binning.bin_tiles(np.array([[32.0, 24.0]]), np.array([[1e6, 1e6]]), np.ones(1), 64, 48, 16, 16)
    assert ((k >> np.uint64(32)).tolist() == list(range(12)))
    assert (r[:, 1] - r[:, 0] == 1).all()
    # ragged image: 70 px with 16-px tiles -> 5 tile columns
    k, i, r = binning.bin_tiles(np.array([[69.5, 1.0]]), np.array([[0.25, 0.25]]), np.ones(1), 70, 20, 16, 16)
    assert (k >> np.uint64(32)).tolist() == [4]
