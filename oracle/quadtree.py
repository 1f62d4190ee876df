"""FP64 reference of the per-frame seeding of new Gaussians (Sec. III-B.2,
Eq. 10): the contrast quadtree over the RGB frame and the back-projection of
its leaf centres.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Definition followed, with the readings where the paper is silent:

* The frame is covered by a grid of square root cells of ``max_size`` px
  (``max_size`` and ``min_size`` powers of two),
  cells clipped at the image border.  A cell splits into its four quadrants
  (each clipped, empty ones dropped) while the mean over the three channels of
  the per-channel variance of its pixels exceeds ``var_thr`` (the paper's
  threshold 0.1 read as a standard deviation, so var_thr = 0.01), its side is
  larger than ``min_size`` and it holds more than one pixel.  Every cell that
  does not split is a leaf.
* A leaf (x0, y0, w, h) is seeded at its centre u = (x0 + w/2, y0 + h/2), read
  at pixel (min(floor(u_x), W-1), min(floor(u_y), H-1)); it is seeded only if
  the depth there is > 0 and, when a coverage image is given, the rendered
  alpha there is below the novelty threshold (0.5).
* Eq. 10: p_c = ((u_x - cx) z / fx, (u_y - cy) z / fy, z), p_w = R^T (p_c - t)
  for the world-to-camera pose (R, t).  Scale d = (w^2 + h^2)^(1/2) / 2 * z / fx
  on all three axes (the back-projected half diagonal), rotation identity,
  opacity 0.5 (logit 0), SH DC coefficients (c - 0.5) / Y_00 so that the
  decoded colour is the pixel colour, higher bands 0.

The variance of a cell is computed directly from its pixels (two passes:
mean, then mean squared deviation), not from integral images.
"""
from __future__ import annotations

import numpy as np

Y00 = 0.5 / np.sqrt(np.pi)


def cell_variance(rgb: np.ndarray, x0: int, y0: int, x1: int, y1: int) -> float:
    """Mean over channels of the variance of rgb[y0:y1, x0:x1, c]."""
    block = np.asarray(rgb[y0:y1, x0:x1, :], np.float64).reshape(-1, 3)
    mu = block.mean(0)
    return float(((block - mu) ** 2).mean(0).mean())


def leaves(rgb: np.ndarray, var_thr: float = 0.01, max_size: int = 64, min_size: int = 1) -> np.ndarray:
    """Leaves as an int64 array [L, 4] of (x0, y0, w, h), in depth-first order."""
    H, W = rgb.shape[:2]
    out = []

    def visit(x0, y0, size):
        x1, y1 = min(x0 + size, W), min(y0 + size, H)
        if x1 <= x0 or y1 <= y0:
            return
        area = (x1 - x0) * (y1 - y0)
        if size > min_size and area > 1 and cell_variance(rgb, x0, y0, x1, y1) > var_thr:
            half = size // 2
            for dy in (0, half):
                for dx in (0, half):
                    visit(x0 + dx, y0 + dy, half)
        else:
            out.append((x0, y0, x1 - x0, y1 - y0))

    for y in range(0, H, max_size):
        for x in range(0, W, max_size):
            visit(x, y, max_size)
    return np.array(out, np.int64).reshape(-1, 4)


def seed(rgb: np.ndarray, depth: np.ndarray, lv: np.ndarray, cam, R_cw, t_cw, sh_degree: int,
         alpha: np.ndarray | None = None, alpha_thr: float = 0.5) -> dict:
    """Eq. 10 for every leaf that passes the depth and coverage tests."""
    H, W = depth.shape
    R = np.asarray(R_cw, np.float64)
    t = np.asarray(t_cw, np.float64)
    means, ls, sh = [], [], []
    K = (sh_degree + 1) ** 2
    for x0, y0, w, h in np.asarray(lv, np.int64):
        ux, uy = x0 + w / 2.0, y0 + h / 2.0
        pi, pj = min(int(np.floor(ux)), W - 1), min(int(np.floor(uy)), H - 1)
        z = float(depth[pj, pi])
        if not z > 0.0:
            continue
        if alpha is not None and not float(alpha[pj, pi]) < alpha_thr:
            continue
        pc = np.array([(ux - cam.cx) * z / cam.fx, (uy - cam.cy) * z / cam.fy, z])
        means.append(R.T @ (pc - t))
        ls.append(np.log(0.5 * np.hypot(w, h) * z / cam.fx))
        coeff = np.zeros((K, 3))
        coeff[0] = (np.asarray(rgb[pj, pi], np.float64) - 0.5) / Y00
        sh.append(coeff)
    n = len(means)
    quats = np.zeros((n, 4))
    quats[:, 0] = 1.0
    return {"means": np.array(means).reshape(n, 3), "log_scales": np.repeat(np.array(ls).reshape(n, 1), 3, 1),
            "quats": quats, "opacity_logits": np.zeros(n), "sh": np.array(sh).reshape(n, K, 3),
            "sh_degree": sh_degree}
