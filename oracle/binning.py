"""Integer tile binning: (tile, depth) keys, stable sort, per-tile ranges.

Test infrastructure.  The paper's rasterizer "divides the screen into
multiple tiles" and sorts the Gaussians "based on depth in each tile"
(Sec. III-B.3).  The rule below is the integer contract the GPU binning
stage must reproduce bit for bit, given float32 inputs per Gaussian:

* mean2d (mx, my), half-extents (ex, ey) of the pixel-space support box and
  camera depth z; a Gaussian takes part iff ex > 0 and ey > 0.
* TX = ceil(W / tw), TY = ceil(H / th) tiles; with float32 arithmetic
  (each operation rounded to nearest) and tw, th powers of two,
      x0 = clamp(floor((mx - ex) * (1/tw)), 0, TX)
      x1 = clamp(floor((mx + ex) * (1/tw)) + 1, 0, TX)       (same for y)
  and the Gaussian is listed in every tile (tx, ty) of [x0, x1) x [y0, y1).
* key = (ty * TX + tx) << 32 | float32 bit pattern of z (z > 0, so the bit
  pattern orders like the value); pairs are emitted Gaussian by Gaussian in
  index order and row-major tile order, then stably sorted by key, so equal
  depths keep index order.
* range[t] = [first, last + 1) of tile t in the sorted list, (0, 0) if empty.

Written with numpy float32 scalars/arrays (IEEE round-to-nearest per
operation, no fused multiply-add) and a stable argsort.
"""
from __future__ import annotations

import numpy as np


def tile_rects(mean2d, extent, width: int, height: int, tile_w: int, tile_h: int):
    m = np.asarray(mean2d, np.float32)
    e = np.asarray(extent, np.float32)
    TX = -(-width // tile_w)
    TY = -(-height // tile_h)
    itw = np.float32(1.0 / tile_w)
    ith = np.float32(1.0 / tile_h)
    lo_x = np.floor((m[:, 0] - e[:, 0]) * itw)
    hi_x = np.floor((m[:, 0] + e[:, 0]) * itw) + np.float32(1.0)
    lo_y = np.floor((m[:, 1] - e[:, 1]) * ith)
    hi_y = np.floor((m[:, 1] + e[:, 1]) * ith) + np.float32(1.0)
    x0 = np.clip(lo_x, 0, TX).astype(np.int64)
    x1 = np.clip(hi_x, 0, TX).astype(np.int64)
    y0 = np.clip(lo_y, 0, TY).astype(np.int64)
    y1 = np.clip(hi_y, 0, TY).astype(np.int64)
    part = (e[:, 0] > 0) & (e[:, 1] > 0)
    x1 = np.where(part, x1, x0)
    y1 = np.where(part, y1, y0)
    return x0, y0, x1, y1, TX, TY


def bin_tiles(mean2d, extent, depth, width: int, height: int, tile_w: int, tile_h: int):
    """Return (keys uint64 [P], ids uint32 [P], ranges uint32 [TX*TY, 2])."""
    x0, y0, x1, y1, TX, TY = tile_rects(mean2d, extent, width, height, tile_w, tile_h)
    zbits = np.asarray(depth, np.float32).view(np.uint32).astype(np.uint64)
    keys, ids = [], []
    for g in range(x0.shape[0]):
        if x1[g] <= x0[g] or y1[g] <= y0[g]:
            continue
        ty, tx = np.meshgrid(np.arange(y0[g], y1[g]), np.arange(x0[g], x1[g]), indexing="ij")
        t = (ty * TX + tx).ravel().astype(np.uint64)
        keys.append((t << np.uint64(32)) | zbits[g])
        ids.append(np.full(t.size, g, np.uint32))
    if keys:
        keys = np.concatenate(keys)
        ids = np.concatenate(ids)
    else:
        keys = np.zeros(0, np.uint64)
        ids = np.zeros(0, np.uint32)
    order = np.argsort(keys, kind="stable")
    keys, ids = keys[order], ids[order]
    T = TX * TY
    ranges = np.zeros((T, 2), np.uint32)
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    if tiles.size:
        starts = np.flatnonzero(np.r_[True, tiles[1:] != tiles[:-1]])
        ends = np.r_[starts[1:], tiles.size]
        ranges[tiles[starts], 0] = starts
        ranges[tiles[starts], 1] = ends
    return keys, ids, ranges
