"""Contrast quadtree seeding of new Gaussians (Sec. III-B.2, Eq. 10).

Each RGB frame is covered by a grid of root cells (64 px); a cell splits into
four while the mean of its per-channel RGB variances exceeds ``var_thr``
(0.01, i.e. a standard deviation of 0.1, the paper's quadtree threshold of
Sec. IV-A.4) and it is larger than ``min_size`` px.  Cells are clipped at the
image border.  Every leaf with valid depth becomes one Gaussian:

* mean: the leaf centre back-projected with the depth at that pixel (Eq. 10),
* rotation R = I (quaternion (1, 0, 0, 0)), scale S = diag(d, d, d) with d the
  back-projected distance from the leaf centre to its corners,
* opacity 0.5 (logit 0), SH DC coefficients set so that the decoded colour is
  the pixel colour at the leaf centre; higher SH bands 0.

Variance is evaluated with integral images of I and I^2 (float64), one level
of the tree at a time.
"""
from __future__ import annotations

import numpy as np

from .scene import Camera, Pose

Y00 = 0.28209479177387814  # 1 / (2 sqrt(pi)), the degree-0 real SH constant


def _integral(a: np.ndarray) -> np.ndarray:
    s = np.zeros((a.shape[0] + 1, a.shape[1] + 1) + a.shape[2:], np.float64)
    s[1:, 1:] = np.cumsum(np.cumsum(a, 0), 1)
    return s


def quadtree_leaves(rgb: np.ndarray, var_thr: float = 0.01, max_size: int = 64, min_size: int = 1):
    """Return leaves as an int array [L, 4] of (x0, y0, w, h) (clipped cells)."""
    H, W = rgb.shape[:2]
    I1 = _integral(rgb.astype(np.float64))
    I2 = _integral(rgb.astype(np.float64) ** 2)
    ys, xs = np.meshgrid(np.arange(0, H, max_size), np.arange(0, W, max_size), indexing="ij")
    cells = np.stack([xs.ravel(), ys.ravel()], 1)
    size = max_size
    leaves = []
    while cells.shape[0]:
        x0, y0 = cells[:, 0], cells[:, 1]
        x1, y1 = np.minimum(x0 + size, W), np.minimum(y0 + size, H)
        keep = (x1 > x0) & (y1 > y0)
        x0, y0, x1, y1 = x0[keep], y0[keep], x1[keep], y1[keep]
        area = ((x1 - x0) * (y1 - y0)).astype(np.float64)

        def box(S):
            return S[y1, x1] - S[y0, x1] - S[y1, x0] + S[y0, x0]

        m1 = box(I1) / area[:, None]
        m2 = box(I2) / area[:, None]
        var = np.maximum(m2 - m1 * m1, 0.0).mean(1)
        split = (var > var_thr) & (size > min_size) & (area > 1)
        leaf = ~split
        leaves.append(np.stack([x0[leaf], y0[leaf], x1[leaf] - x0[leaf], y1[leaf] - y0[leaf]], 1))
        half = size // 2
        sx, sy = x0[split], y0[split]
        cells = np.concatenate([np.stack([sx, sy], 1), np.stack([sx + half, sy], 1),
                                np.stack([sx, sy + half], 1), np.stack([sx + half, sy + half], 1)])
        size = half
        if size < min_size:
            break
    return np.concatenate(leaves).astype(np.int64)


def seed_gaussians(rgb: np.ndarray, depth: np.ndarray, cam: Camera, pose: Pose, sh_degree: int,
                   var_thr: float = 0.01, max_size: int = 64, min_size: int = 1, mask: np.ndarray | None = None):
    """Quadtree-seed Gaussians from one RGB-D frame; returns a parameter dict.
    ``mask`` [H, W] (optional): only leaves whose centre pixel is True are
    seeded (the novelty rule of the per-frame loop)."""
    leaves = quadtree_leaves(rgb, var_thr, max_size, min_size)
    x0, y0, w, h = leaves.T
    uc = x0 + w / 2.0
    vc = y0 + h / 2.0
    pi = np.minimum(np.floor(uc).astype(np.int64), cam.width - 1)
    pj = np.minimum(np.floor(vc).astype(np.int64), cam.height - 1)
    z = depth[pj, pi].astype(np.float64)
    ok = z > 0
    if mask is not None:
        ok &= np.asarray(mask, bool)[pj, pi]
    uc, vc, z, w, h, pi, pj = uc[ok], vc[ok], z[ok], w[ok], h[ok], pi[ok], pj[ok]
    pc = np.stack([(uc - cam.cx) * z / cam.fx, (vc - cam.cy) * z / cam.fy, z], 1)
    pw = (pc - pose.t.astype(np.float64)[None]) @ pose.R.astype(np.float64)  # R^T (p_c - t)
    d = 0.5 * np.sqrt(w.astype(np.float64) ** 2 + h.astype(np.float64) ** 2) * z / cam.fx
    n = pw.shape[0]
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n, K, 3), np.float32)
    sh[:, 0, :] = (rgb[pj, pi].astype(np.float64) - 0.5) / Y00
    quats = np.zeros((n, 4), np.float32)
    quats[:, 0] = 1.0
    return {
        "means": pw.astype(np.float32),
        "log_scales": np.repeat(np.log(d)[:, None], 3, 1).astype(np.float32),
        "quats": quats,
        "opacity_logits": np.zeros(n, np.float32),
        "sh": sh,
        "sh_degree": sh_degree,
    }
