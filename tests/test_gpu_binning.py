"""Tile binning on the GPU (gs_bin_tiles) is bit-exact against the integer
binning oracle: keys, ids and per-tile ranges."""
import numpy as np
import pytest
import torch

from oracle import binning
from tests._util import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    ensure_built()
    from paper_2408_12677_gb300.torch_api import Context
    c = Context(0)
    yield c
    c.close()


def _run(ctx, mean2d, extent, depth, W, H, tw, th):
    from paper_2408_12677_gb300 import abi
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")
    TX, TY = -(-W // tw), -(-H // th)
    ranges = torch.zeros((TX * TY, 2), dtype=torch.int32, device="cuda")
    P = abi.gs_bin_tiles(ctx.handle, t(mean2d), t(extent), t(depth), W, H, tw, th, None, None, ranges)
    if P < -1:
        P = -P - 1
    keys = torch.zeros(max(P, 1), dtype=torch.int64, device="cuda")
    ids = torch.zeros(max(P, 1), dtype=torch.int32, device="cuda")
    P2 = abi.gs_bin_tiles(ctx.handle, t(mean2d), t(extent), t(depth), W, H, tw, th, keys, ids, ranges)
    assert P2 == P
    return (keys[:P].cpu().numpy().view(np.uint64), ids[:P].cpu().numpy().view(np.uint32),
            ranges.cpu().numpy().view(np.uint32))


def _case(rng, n, W, H, max_ext, ties=False):
    mean2d = np.stack([rng.uniform(-0.1 * W, 1.1 * W, n), rng.uniform(-0.1 * H, 1.1 * H, n)], 1).astype(np.float32)
    extent = rng.uniform(0.2, max_ext, (n, 2)).astype(np.float32)
    extent[rng.uniform(0, 1, n) < 0.05] = 0.0  # culled
    depth = (rng.integers(1, 8, n) * 0.25 if ties else rng.uniform(0.2, 8.0, n)).astype(np.float32)
    return mean2d, extent, depth


@pytest.mark.parametrize("tw,th", [(16, 16), (8, 32), (32, 8)])
@pytest.mark.parametrize("W,H,n,max_ext,ties", [(64, 48, 500, 20.0, False), (100, 70, 3000, 12.0, True),
                                                 (1200, 680, 60000, 40.0, False),
                                                 # more than 4096 tiles: the multi-block scan, a ragged last block
                                                 (2600, 1950, 90000, 30.0, True)])
def test_bitexact(ctx, tw, th, W, H, n, max_ext, ties):
    rng = np.random.default_rng(W * 7 + n + tw)
    m, e, z = _case(rng, n, W, H, max_ext, ties)
    keys, ids, ranges = _run(ctx, m, e, z, W, H, tw, th)
    rk, ri, rr = binning.bin_tiles(m, e, z, W, H, tw, th)
    assert keys.size == rk.size
    np.testing.assert_array_equal(keys, rk)
    np.testing.assert_array_equal(ids, ri)
    np.testing.assert_array_equal(ranges, rr)


def test_edge_cases(ctx):
    # empty input
    keys, ids, ranges = _run(ctx, np.zeros((0, 2)), np.zeros((0, 2)), np.zeros(0), 64, 48, 16, 16)
    assert keys.size == 0 and not ranges.any()
    # nothing on screen
    m = np.array([[-500.0, 10.0], [10.0, 900.0]])
    keys, ids, ranges = _run(ctx, m, np.full((2, 2), 3.0), np.ones(2), 64, 48, 16, 16)
    assert keys.size == 0
    # one Gaussian covering a 1x1-tile image; and a huge one over a ragged image
    keys, ids, ranges = _run(ctx, np.array([[4.0, 4.0]]), np.array([[100.0, 100.0]]), np.ones(1), 8, 8, 16, 16)
    assert keys.tolist() == [(0 << 32) | int(np.float32(1).view(np.uint32))] and ranges.tolist() == [[0, 1]]
    rng = np.random.default_rng(1)
    m, e, z = _case(rng, 200, 333, 77, 400.0)
    k1, i1, r1 = _run(ctx, m, e, z, 333, 77, 16, 16)
    rk, ri, rr = binning.bin_tiles(m, e, z, 333, 77, 16, 16)
    np.testing.assert_array_equal(k1, rk)
    np.testing.assert_array_equal(i1, ri)
    np.testing.assert_array_equal(r1, rr)


def test_long_tile_lists_take_the_radix_fallback(ctx):
    """Tile lists longer than the per-tile shared-memory sort holds (4096)
    switch the whole frame to the radix-sort binning; still bit-exact."""
    rng = np.random.default_rng(77)
    n = 6000
    m = np.stack([rng.uniform(0, 64, n), rng.uniform(0, 48, n)], 1).astype(np.float32)
    e = np.full((n, 2), 200.0, np.float32)  # every Gaussian covers all 12 tiles
    z = (rng.integers(1, 50, n) * 0.1).astype(np.float32)
    keys, ids, ranges = _run(ctx, m, e, z, 64, 48, 16, 16)
    rk, ri, rr = binning.bin_tiles(m, e, z, 64, 48, 16, 16)
    assert (rr[:, 1] - rr[:, 0]).max() > 4096
    np.testing.assert_array_equal(keys, rk)
    np.testing.assert_array_equal(ids, ri)
    np.testing.assert_array_equal(ranges, rr)


@pytest.mark.parametrize("L", [2, 3, 31, 32, 33, 64, 65, 128, 129, 255, 256, 257, 511, 512, 513, 1000, 4096])
def test_list_lengths_of_every_sort_path(ctx, L):
    """Lists of exactly L entries in tile 0 and L // 2 + 1 in tile 1 of a
    two-tile image: both register widths of the per-warp sort (up to 256
    and 512 entries, short lists padded), the CTA-wide sort beyond 512 and
    its limit of 4096; depths drawn from few values so that ties are broken
    by id."""
    rng = np.random.default_rng(L)
    n0, n1 = L, L // 2 + 1
    m = np.concatenate([np.stack([rng.uniform(2, 14, n0), rng.uniform(2, 14, n0)], 1),
                        np.stack([rng.uniform(18, 30, n1), rng.uniform(2, 14, n1)], 1)]).astype(np.float32)
    e = np.full((n0 + n1, 2), 1.5, np.float32)  # stays inside its tile
    z = (rng.integers(1, 9, n0 + n1) * 0.5).astype(np.float32)
    perm = rng.permutation(n0 + n1)  # ids of the two tiles interleaved
    m, e, z = m[perm], e[perm], z[perm]
    keys, ids, ranges = _run(ctx, m, e, z, 32, 16, 16, 16)
    rk, ri, rr = binning.bin_tiles(m, e, z, 32, 16, 16, 16)
    assert (rr[:, 1] - rr[:, 0]).tolist() == [n0, n1]
    np.testing.assert_array_equal(keys, rk)
    np.testing.assert_array_equal(ids, ri)
    np.testing.assert_array_equal(ranges, rr)
