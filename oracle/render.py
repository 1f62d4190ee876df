"""FP64 reference rasterizer: projection, untiled compositing, loss, gradients.

Test infrastructure (see ``oracle/__init__.py``).  Everything is float64 torch
on the CPU; gradients come from torch.autograd through this forward
definition, so the oracle's gradient *is* the derivative of the function
below (pinned against central finite differences in the tests).

Definition followed (Sec. III-A.2 Eq. 1-5, Sec. III-B.3 Eq. 11-12), with the
readings where the paper is silent:

* Gaussian g: mean p_g, rotation R from the normalised quaternion (w, x, y, z),
  scale S = diag(exp(log_s)), covariance Sigma = R S S^T R^T (Eq. 2), opacity
  sigmoid(logit), SH colour coefficients (``oracle.sh``).
* Camera: world-to-camera T_CW = T_WC^{-1} = (W, t); p_c = W p_g + t (Eq. 4);
  pi(p_c) = (fx x/z + cx, fy y/z + cy); pixel (i, j) has its centre at
  (i + 0.5, j + 0.5).  Gaussians with z <= near (0.2 m) are culled.
* 2D covariance (Eq. 5): Sigma^ = J W Sigma W^T J^T + 0.3 I, with J the
  Jacobian of pi at p_c evaluated at x~ = z clamp(x/z, -1.3 W/(2 fx),
  1.3 W/(2 fx)) (same for y); conic = Sigma^^{-1}.
* Colour c_g = max(0, 0.5 + sum_k Y_k(d) k_gk) with d the unit vector from
  the camera centre -W^T t to p_g.
* Compositing (Eq. 11) at pixel centre u over the Gaussians ordered by
  (float32(z), index): q = (u - mu)^T conic (u - mu); a Gaussian takes part iff
  q <= 9 and alpha = min(0.99, opacity * exp(-q/2)) >= 1/255; blending stops
  before the first taking-part Gaussian with T (1 - alpha) < 1e-4.
  colour = sum c_i alpha_i T_i + T_final bg, depth = sum z_i alpha_i T_i,
  alpha image = 1 - T_final.
* Loss (Eq. 12 plus a depth term): 0.8 mean|C^ - C| over 3HW values plus
  0.2 mean|D^ - D| over pixels whose target depth is > 0.

No tiling: every Gaussian is tested at every requested pixel ("brute" mode).
The "prefilter" mode first drops, per chunk of pixels, Gaussians whose q
exceeds 9 at every pixel of the chunk (they contribute exactly nothing); the
tests check that both modes agree bit for bit.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from .sh import sh_to_rgb

DT = torch.float64


@dataclasses.dataclass
class RasterCfg:
    near: float = 0.2
    dilation: float = 0.3
    q_max: float = 9.0
    alpha_max: float = 0.99
    alpha_min: float = 1.0 / 255.0
    t_eps: float = 1e-4
    bg: tuple = (0.0, 0.0, 0.0)
    frustum_clamp: float = 1.3


@dataclasses.dataclass
class LossCfg:
    w_color: float = 0.8
    w_depth: float = 0.2


PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


def to_tensors(params: dict, requires_grad: bool = False) -> dict:
    """float32 numpy parameter dict -> float64 torch leaves."""
    out = {}
    for k in PARAM_NAMES:
        t = torch.as_tensor(np.asarray(params[k]), dtype=DT).clone()
        t.requires_grad_(requires_grad)
        out[k] = t
    return out


# ----------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------
def quat_to_rotmat(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrix of the normalised quaternion q = (w, x, y, z)."""
    q = q / torch.linalg.vector_norm(q, dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    rows = [
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y),
    ]
    return torch.stack(rows, -1).reshape(q.shape[:-1] + (3, 3))


def covariance_3d(log_scales: torch.Tensor, quats: torch.Tensor) -> torch.Tensor:
    """Sigma = R S S^T R^T (Eq. 2)."""
    R = quat_to_rotmat(quats)
    M = R * torch.exp(log_scales)[..., None, :]  # R @ diag(s)
    return M @ M.transpose(-1, -2)


def se3_exp(xi: torch.Tensor) -> torch.Tensor:
    """4x4 exp of the twist xi = (rho, phi) (matrix exponential of xi^)."""
    rho, phi = xi[:3], xi[3:]
    z = torch.zeros((), dtype=xi.dtype)
    A = torch.stack([
        torch.stack([z, -phi[2], phi[1], rho[0]]),
        torch.stack([phi[2], z, -phi[0], rho[1]]),
        torch.stack([-phi[1], phi[0], z, rho[2]]),
        torch.stack([z, z, z, z]),
    ])
    return torch.linalg.matrix_exp(A)


def perturb_pose(R_cw: torch.Tensor, t_cw: torch.Tensor, xi: torch.Tensor):
    """Left perturbation T_CW(xi) = exp(xi^) T_CW."""
    E = se3_exp(xi)
    return E[:3, :3] @ R_cw, E[:3, :3] @ t_cw + E[:3, 3]


def project(P: dict, sh_degree: int, cam, R_cw: torch.Tensor, t_cw: torch.Tensor,
            cfg: RasterCfg = RasterCfg()) -> dict:
    """Per-Gaussian 2D quantities for the Gaussians that survive culling."""
    R_cw = torch.as_tensor(R_cw, dtype=DT)
    t_cw = torch.as_tensor(t_cw, dtype=DT)
    means = P["means"]
    with torch.no_grad():
        z_all = means @ R_cw[2] + t_cw[2]
    idx = torch.nonzero(z_all > cfg.near).flatten()
    p = means[idx]
    pc = p @ R_cw.T + t_cw
    x, y, z = pc.unbind(-1)
    fx, fy, cx, cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    mu = torch.stack([fx * x / z + cx, fy * y / z + cy], -1)

    Sigma = covariance_3d(P["log_scales"][idx], P["quats"][idx])
    Sp = R_cw @ Sigma @ R_cw.T
    limx = cfg.frustum_clamp * float(cam.width) / (2.0 * fx)
    limy = cfg.frustum_clamp * float(cam.height) / (2.0 * fy)
    xt = z * torch.clamp(x / z, -limx, limx)
    yt = z * torch.clamp(y / z, -limy, limy)
    zero = torch.zeros_like(z)
    J = torch.stack([
        torch.stack([fx / z, zero, -fx * xt / (z * z)], -1),
        torch.stack([zero, fy / z, -fy * yt / (z * z)], -1),
    ], -2)
    cov2d = J @ Sp @ J.transpose(-1, -2) + cfg.dilation * torch.eye(2, dtype=DT)
    a, b, c = cov2d[:, 0, 0], cov2d[:, 0, 1], cov2d[:, 1, 1]
    det = a * c - b * b
    keep = det > 0
    conic = torch.stack([c / det, -b / det, a / det], -1)

    cam_center = -(R_cw.T @ t_cw)
    d = p - cam_center
    dirs = d / torch.linalg.vector_norm(d, dim=-1, keepdim=True)
    rgb = sh_to_rgb(P["sh"][idx], dirs, sh_degree)
    opac = torch.sigmoid(P["opacity_logits"][idx])

    sel = torch.nonzero(keep).flatten()
    out = {
        "idx": idx[sel], "mean2d": mu[sel], "cov2d": cov2d[sel], "conic": conic[sel],
        "depth": z[sel], "rgb": rgb[sel], "opacity": opac[sel],
    }
    # compositing order: float32 depth, then Gaussian index (stable)
    z32 = out["depth"].detach().numpy().astype(np.float32)
    order = np.lexsort((out["idx"].numpy(), z32))
    out["order"] = torch.as_tensor(order, dtype=torch.long)
    return out


# ----------------------------------------------------------------------------
# compositing
# ----------------------------------------------------------------------------
def _quad_form(U: torch.Tensor, mu: torch.Tensor, conic: torch.Tensor) -> torch.Tensor:
    d = U[:, None, :] - mu[None, :, :]
    dx, dy = d[..., 0], d[..., 1]
    return conic[None, :, 0] * dx * dx + 2.0 * conic[None, :, 1] * dx * dy + conic[None, :, 2] * dy * dy


def _composite_chunk(U, mu, conic, opac, rgb, z, cfg: RasterCfg):
    q = _quad_form(U, mu, conic)
    G = torch.exp(-0.5 * q)
    alpha = torch.clamp(opac[None, :] * G, max=cfg.alpha_max)
    active = (q <= cfg.q_max) & (alpha >= cfg.alpha_min)
    a = torch.where(active, alpha, torch.zeros_like(alpha))
    one_minus = 1.0 - a
    T_incl = torch.cumprod(one_minus, dim=1)
    added = active & (T_incl >= cfg.t_eps)
    T_excl = torch.cat([torch.ones_like(T_incl[:, :1]), T_incl[:, :-1]], 1)
    w = torch.where(added, a * T_excl, torch.zeros_like(a))
    T_final = torch.prod(torch.where(added, one_minus, torch.ones_like(one_minus)), 1)
    bg = torch.tensor(cfg.bg, dtype=DT)
    color = w @ rgb + T_final[:, None] * bg[None]
    depth = w @ z
    return color, depth, T_final, added.sum(1)


def pixel_centers(cam) -> torch.Tensor:
    jj, ii = torch.meshgrid(torch.arange(cam.height, dtype=DT), torch.arange(cam.width, dtype=DT), indexing="ij")
    return torch.stack([ii.flatten() + 0.5, jj.flatten() + 0.5], -1)


def _pixel_chunks(U: torch.Tensor, mu, conic, cov, cfg: RasterCfg, prefilter, chunk_elems: int, chunk_px):
    """The pixel chunks of ``composite`` / ``decision_margins``: yields
    (start, stop, use) with ``use`` None (every Gaussian) or the indices of
    the Gaussians kept for the chunk (see ``composite``)."""
    n, M = mu.shape[0], U.shape[0]
    if prefilter == "bbox":
        sizes = [chunk_px] * (-(-M // chunk_px)) if isinstance(chunk_px, int) else list(chunk_px)
        # the box of q <= 9 (1 + 1e-3): also every pair that decision_margins
        # counts as near the support (keeping more Gaussians changes nothing)
        qb = cfg.q_max * (1 + 1e-3)
        ext = torch.stack([torch.sqrt(qb * cov[:, 0, 0]), torch.sqrt(qb * cov[:, 1, 1])], -1)
        ext = ext * (1 + 1e-9) + 1e-9
    else:
        step = max(1, chunk_elems // max(n, 1))
        sizes = [step] * (-(-M // step))
    s0 = 0
    for size in sizes:
        Uc = U[s0:s0 + size]
        use = None
        if prefilter == "bbox" and n > 0:
            lo, hi = Uc.min(0).values, Uc.max(0).values
            gap = torch.maximum(lo[None] - mu, mu - hi[None]).clamp(min=0.0)
            use = torch.nonzero((gap <= ext).all(1)).flatten()
        elif prefilter and n > 0:
            use = torch.nonzero((_quad_form(Uc, mu, conic) <= cfg.q_max).any(0)).flatten()
        yield s0, s0 + Uc.shape[0], use
        s0 += size


def composite(proj: dict, U: torch.Tensor, cfg: RasterCfg = RasterCfg(), prefilter=False,
              chunk_elems: int = 1 << 21, chunk_px=256):
    """Front-to-back compositing at pixel centres U [M, 2] (Eq. 11), no tiling.

    ``prefilter``: False evaluates every Gaussian at every pixel; True drops,
    per chunk of pixels, the Gaussians whose q exceeds 9 at every pixel of
    the chunk; "bbox" takes the pixels ``chunk_px`` at a time (an int, or
    a list of group sizes: pass them grouped by image region, e.g. the tiles
    of ``tile_pixels``) and keeps the Gaussians whose q <= 9 (1 + 1e-3)
    ellipse's bounding box, mu +- sqrt(9.009 diag Sigma^), meets the chunk's
    bounding box -- the others have q > 9 at every pixel of the chunk.  Dropped Gaussians
    contribute exactly nothing, so all three give the same values."""
    o = proj["order"]
    mu, conic, opac = proj["mean2d"][o], proj["conic"][o], proj["opacity"][o]
    rgb, z = proj["rgb"][o], proj["depth"][o]
    M = U.shape[0]
    if M == 0:
        return (torch.zeros((0, 3), dtype=DT), torch.zeros(0, dtype=DT), torch.zeros(0, dtype=DT),
                torch.zeros(0, dtype=torch.long))
    cols, deps, Ts, ns = [], [], [], []
    with torch.no_grad():
        chunks = list(_pixel_chunks(U, mu.detach(), conic.detach(), proj["cov2d"][o].detach(), cfg, prefilter,
                                    chunk_elems, chunk_px))
    for s0, s1, use in chunks:
        Uc = U[s0:s1]
        if use is None:
            c, d, T, k = _composite_chunk(Uc, mu, conic, opac, rgb, z, cfg)
        else:
            c, d, T, k = _composite_chunk(Uc, mu[use], conic[use], opac[use], rgb[use], z[use], cfg)
        cols.append(c)
        deps.append(d)
        Ts.append(T)
        ns.append(k)
    return torch.cat(cols), torch.cat(deps), torch.cat(Ts), torch.cat(ns)


def tile_pixels(cam, tiles, tile_w: int = 16, tile_h: int = 16, sizes: bool = False):
    """Integer (i, j) pixel coordinates [M, 2] of the listed tiles (tile
    index = ty * tiles_x + tx), tile by tile, clipped to the image; with
    ``sizes`` also the pixel count of each tile (pass both to ``render``
    with prefilter="bbox" and chunk_px = the counts)."""
    tx = -(-cam.width // tile_w)
    out, counts = [], []
    for t in tiles:
        x0, y0 = (int(t) % tx) * tile_w, (int(t) // tx) * tile_h
        jj, ii = np.meshgrid(np.arange(y0, min(y0 + tile_h, cam.height)),
                             np.arange(x0, min(x0 + tile_w, cam.width)), indexing="ij")
        out.append(np.stack([ii.ravel(), jj.ravel()], 1))
        counts.append(out[-1].shape[0])
    pix = np.concatenate(out) if out else np.zeros((0, 2), np.int64)
    return (pix, counts) if sizes else pix


def render(P: dict, sh_degree: int, cam, R_cw, t_cw, cfg: RasterCfg = RasterCfg(), pixels=None,
           prefilter=False, chunk_px=256) -> dict:
    """Render colour [3, M], depth [M], alpha [M] (M = H*W unless ``pixels``
    [M, 2] integer (i, j) coordinates are given).  Full images are reshaped to
    [3, H, W] / [H, W]."""
    proj = project(P, sh_degree, cam, R_cw, t_cw, cfg)
    if pixels is None:
        U = pixel_centers(cam)
    else:
        U = torch.as_tensor(np.asarray(pixels), dtype=DT) + 0.5
    color, depth, T, ncon = composite(proj, U, cfg, prefilter, chunk_px=chunk_px)
    out = {"color": color.T.contiguous(), "depth": depth, "alpha": 1.0 - T, "T_final": T, "n_contrib": ncon}
    if pixels is None:
        H, W = cam.height, cam.width
        out = {"color": out["color"].reshape(3, H, W), "depth": depth.reshape(H, W),
               "alpha": out["alpha"].reshape(H, W), "T_final": T.reshape(H, W),
               "n_contrib": ncon.reshape(H, W)}
    out["proj"] = proj
    return out


# ----------------------------------------------------------------------------
# loss (Eq. 12 plus the depth term)
# ----------------------------------------------------------------------------
def loss_l1(color, depth, target_rgb, target_depth, cfg: LossCfg = LossCfg()):
    target_rgb = torch.as_tensor(np.asarray(target_rgb), dtype=DT)
    target_depth = torch.as_tensor(np.asarray(target_depth), dtype=DT)
    lc = torch.abs(color - target_rgb).sum() / color.numel()
    valid = target_depth > 0
    nv = int(valid.sum())
    ld = torch.where(valid, torch.abs(depth - target_depth), torch.zeros_like(depth)).sum() / max(nv, 1)
    return cfg.w_color * lc + cfg.w_depth * ld


def loss_image_grads(color, depth, target_rgb, target_depth, cfg: LossCfg = LossCfg()):
    """dL/dcolor, dL/ddepth of ``loss_l1`` (via autograd)."""
    c = torch.as_tensor(np.asarray(color), dtype=DT).clone().requires_grad_(True)
    d = torch.as_tensor(np.asarray(depth), dtype=DT).clone().requires_grad_(True)
    L = loss_l1(c, d, target_rgb, target_depth, cfg)
    gc, gd = torch.autograd.grad(L, (c, d))
    return L.detach(), gc, gd


def render_loss(P, sh_degree, cam, R_cw, t_cw, target_rgb, target_depth, rcfg=RasterCfg(), lcfg=LossCfg()):
    out = render(P, sh_degree, cam, R_cw, t_cw, rcfg)
    return loss_l1(out["color"], out["depth"], target_rgb, target_depth, lcfg), out


def gradients(params: dict, sh_degree: int, cam, R_cw, t_cw, target_rgb, target_depth,
              rcfg=RasterCfg(), lcfg=LossCfg(), with_pose: bool = True):
    """Loss and its gradient w.r.t. every parameter (and the 6-DoF pose
    xi = (rho, phi) of the left perturbation exp(xi^) T_CW, at xi = 0)."""
    P = to_tensors(params, requires_grad=True)
    R = torch.as_tensor(np.asarray(R_cw), dtype=DT)
    t = torch.as_tensor(np.asarray(t_cw), dtype=DT)
    xi = torch.zeros(6, dtype=DT, requires_grad=True)
    if with_pose:
        R, t = perturb_pose(R, t, xi)
    L, out = render_loss(P, sh_degree, cam, R, t, target_rgb, target_depth, rcfg, lcfg)
    leaves = [P[k] for k in PARAM_NAMES] + ([xi] if with_pose else [])
    g = torch.autograd.grad(L, leaves, allow_unused=True)
    grads = {k: (gi if gi is not None else torch.zeros_like(P[k])) for k, gi in zip(PARAM_NAMES, g)}
    if with_pose:
        grads["pose"] = g[-1] if g[-1] is not None else torch.zeros(6, dtype=DT)
    return L.detach(), grads, out


def weighted_pixel_gradients(params: dict, sh_degree: int, cam, R_cw, t_cw, pixels, w_color, w_depth,
                             w_alpha=None, rcfg=RasterCfg(), with_pose: bool = True, prefilter=True,
                             chunk_px=256):
    """Gradient of sum_s <w_color[:, s], C(u_s)> + w_depth[s] D(u_s) + w_alpha[s] A(u_s)
    over the listed pixels only (a sparse upstream gradient)."""
    P = to_tensors(params, requires_grad=True)
    R = torch.as_tensor(np.asarray(R_cw), dtype=DT)
    t = torch.as_tensor(np.asarray(t_cw), dtype=DT)
    xi = torch.zeros(6, dtype=DT, requires_grad=True)
    if with_pose:
        R, t = perturb_pose(R, t, xi)
    out = render(P, sh_degree, cam, R, t, rcfg, pixels=pixels, prefilter=prefilter, chunk_px=chunk_px)
    obj = (out["color"] * torch.as_tensor(np.asarray(w_color), dtype=DT)).sum()
    obj = obj + (out["depth"] * torch.as_tensor(np.asarray(w_depth), dtype=DT)).sum()
    if w_alpha is not None:
        obj = obj + (out["alpha"] * torch.as_tensor(np.asarray(w_alpha), dtype=DT)).sum()
    leaves = [P[k] for k in PARAM_NAMES] + ([xi] if with_pose else [])
    g = torch.autograd.grad(obj, leaves, allow_unused=True)
    grads = {k: (gi if gi is not None else torch.zeros_like(P[k])) for k, gi in zip(PARAM_NAMES, g)}
    if with_pose:
        grads["pose"] = g[-1] if g[-1] is not None else torch.zeros(6, dtype=DT)
    return grads, out


# ----------------------------------------------------------------------------
# several views of one map (batched multi-view form)
# ----------------------------------------------------------------------------
def multiview_gradients(params: dict, sh_degree: int, cams, poses, targets, rcfg=RasterCfg(), lcfg=LossCfg(),
                        with_pose: bool = True):
    """Objective of one batched iteration over V views of the same map:
    L = sum over v of L_v, L_v the single-view loss of view v (Eq. 12 plus
    the depth term, each normalised by its own pixel count).  The paper
    optimises view by view (Sec. III-B.3); summing the per-view losses is the
    reading under which one batched Adam step uses the gradients of all views
    at once.  Returns L, its gradient w.r.t. every parameter array, the pose
    twist gradient of every view [V, 6] and the per-view renders.
    ``poses`` is a list of (R_cw, t_cw); ``targets`` a list of (rgb, depth)."""
    P = to_tensors(params, requires_grad=True)
    xis = []
    L = torch.zeros((), dtype=DT)
    outs = []
    for cam, (R_cw, t_cw), (trgb, tdep) in zip(cams, poses, targets):
        R = torch.as_tensor(np.asarray(R_cw), dtype=DT)
        t = torch.as_tensor(np.asarray(t_cw), dtype=DT)
        xi = torch.zeros(6, dtype=DT, requires_grad=True)
        xis.append(xi)
        if with_pose:
            R, t = perturb_pose(R, t, xi)
        Lv, out = render_loss(P, sh_degree, cam, R, t, trgb, tdep, rcfg, lcfg)
        L = L + Lv
        outs.append(out)
    leaves = [P[k] for k in PARAM_NAMES] + (xis if with_pose else [])
    g = torch.autograd.grad(L, leaves, allow_unused=True)
    grads = {k: (gi if gi is not None else torch.zeros_like(P[k])) for k, gi in zip(PARAM_NAMES, g)}
    if with_pose:
        grads["pose"] = torch.stack([gi if gi is not None else torch.zeros(6, dtype=DT)
                                     for gi in g[len(PARAM_NAMES):]])
    return L.detach(), grads, outs


def multiview_weighted_gradients(params: dict, sh_degree: int, cams, poses, w_color, w_depth, w_alpha=None,
                                 rcfg=RasterCfg(), with_pose: bool = True, prefilter: bool = True):
    """Gradient of sum over views v and pixels s of <w_color[v][:, s], C_v(u_s)>
    + w_depth[v][s] D_v(u_s) + w_alpha[v][s] A_v(u_s) (full images; the
    upstream gradients of a batched backward pass).  Pose gradients [V, 6]."""
    P = to_tensors(params, requires_grad=True)
    xis = []
    obj = torch.zeros((), dtype=DT)
    for v, (cam, (R_cw, t_cw)) in enumerate(zip(cams, poses)):
        R = torch.as_tensor(np.asarray(R_cw), dtype=DT)
        t = torch.as_tensor(np.asarray(t_cw), dtype=DT)
        xi = torch.zeros(6, dtype=DT, requires_grad=True)
        xis.append(xi)
        if with_pose:
            R, t = perturb_pose(R, t, xi)
        jj, ii = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
        pix = np.stack([ii.ravel(), jj.ravel()], 1)
        out = render(P, sh_degree, cam, R, t, rcfg, pixels=pix, prefilter=prefilter)
        obj = obj + (out["color"] * torch.as_tensor(np.asarray(w_color[v]).reshape(3, -1), dtype=DT)).sum()
        obj = obj + (out["depth"] * torch.as_tensor(np.asarray(w_depth[v]).reshape(-1), dtype=DT)).sum()
        if w_alpha is not None and w_alpha[v] is not None:
            obj = obj + (out["alpha"] * torch.as_tensor(np.asarray(w_alpha[v]).reshape(-1), dtype=DT)).sum()
    leaves = [P[k] for k in PARAM_NAMES] + (xis if with_pose else [])
    g = torch.autograd.grad(obj, leaves, allow_unused=True)
    grads = {k: (gi if gi is not None else torch.zeros_like(P[k])) for k, gi in zip(PARAM_NAMES, g)}
    if with_pose:
        grads["pose"] = torch.stack([gi if gi is not None else torch.zeros(6, dtype=DT)
                                     for gi in g[len(PARAM_NAMES):]])
    return grads


# ----------------------------------------------------------------------------
# distances to the decision thresholds (for the float32 / float64 flip audit)
# ----------------------------------------------------------------------------
MARGIN_KINDS = ("q = 9", "alpha = 1/255", "T (1 - alpha) = 1e-4", "alpha = 0.99", "L1 residual = 0")


def decision_margins(P: dict, sh_degree: int, cam, R_cw, t_cw, cfg: RasterCfg = RasterCfg(), pixels=None,
                     chunk_elems: int = 1 << 21, prefilter=False, chunk_px=256, pixel_extra=None) -> dict:
    """Relative float64 distances of the compositing decisions (Eq. 11 with
    the support, skip, stop and clamp rules) to their thresholds: for a
    (pixel, Gaussian) pair near or inside the support, |q - 9| / 9, and where
    q <= 9, |alpha - 1/255| / (1/255) and |alpha - 0.99| / 0.99 (alpha before
    the clamp); for a pixel, |T (1 - alpha) - 1e-4| / 1e-4 over its active
    Gaussians (those with q <= 9 and alpha >= 1/255).  A float32 evaluation
    can take a decision the other way only where this distance is within its
    rounding error.  Returns per pixel (M = H*W unless ``pixels`` [M, 2]):
    ``pixel`` the smallest distance over its pairs and its stop test,
    ``pixel_kind`` (index into MARGIN_KINDS), ``pixel_gid`` (the Gaussian);
    per Gaussian (parameter index): ``gauss`` the smallest distance over the
    pixels where it is active or near its support, counting each such
    pixel's stop test too (a stop that flips changes the gradient of every
    Gaussian the pixel reaches), and ``gauss_kind``.  ``prefilter`` and
    ``chunk_px`` as in ``composite`` (the bounding box there holds every
    pixel with q <= 9 (1 + 1e-3), so a dropped pair's only decision, q <= 9,
    is more than 1e-3 from its threshold).  ``pixel_extra`` [M] (optional):
    a further per-pixel distance (kind 4, e.g. an L1 loss residual's distance
    to 0, whose sign decides the image gradient) folded into the pixel's
    margin and into every Gaussian the pixel reaches."""
    with torch.no_grad():
        T = to_tensors(P)
        proj = project(T, sh_degree, cam, torch.as_tensor(np.asarray(R_cw), dtype=DT),
                       torch.as_tensor(np.asarray(t_cw), dtype=DT), cfg)
        U = pixel_centers(cam) if pixels is None else torch.as_tensor(np.asarray(pixels), dtype=DT) + 0.5
        o = proj["order"]
        mu, conic, opac = proj["mean2d"][o], proj["conic"][o], proj["opacity"][o]
        gid = proj["idx"][o]
        n, M = mu.shape[0], U.shape[0]
        N = P["means"].shape[0]
        inf = torch.full((), float("inf"), dtype=DT)
        pix = torch.full((M,), float("inf"), dtype=DT)
        pix_kind = torch.zeros(M, dtype=torch.long)
        pix_gid = torch.full((M,), -1, dtype=torch.long)
        gm = torch.full((max(n, 1),), float("inf"), dtype=DT)
        gk = torch.zeros(max(n, 1), dtype=torch.long)
        extra = None if pixel_extra is None else torch.as_tensor(np.asarray(pixel_extra, np.float64)).reshape(-1)
        chunks = list(_pixel_chunks(U, mu, conic, proj["cov2d"][o], cfg, prefilter, chunk_elems, chunk_px)) \
            if n and M else []
        for s0, s1, use in chunks:
            sel = torch.arange(n) if use is None else use
            q = _quad_form(U[s0:s1], mu[sel], conic[sel])
            araw = opac[sel][None, :] * torch.exp(-0.5 * q)
            near = q <= cfg.q_max * (1 + 1e-3)
            inside = q <= cfg.q_max
            m_q = torch.where(near, torch.abs(q - cfg.q_max) / cfg.q_max, inf)
            m_a = torch.where(inside, torch.abs(araw - cfg.alpha_min) / cfg.alpha_min, inf)
            m_c = torch.where(inside, torch.abs(araw - cfg.alpha_max) / cfg.alpha_max, inf)
            alpha = torch.clamp(araw, max=cfg.alpha_max)
            active = inside & (alpha >= cfg.alpha_min)
            a = torch.where(active, alpha, torch.zeros_like(alpha))
            T_incl = torch.cumprod(1.0 - a, dim=1)
            T_excl = torch.cat([torch.ones_like(T_incl[:, :1]), T_incl[:, :-1]], 1)
            m_t = torch.where(active, torch.abs(T_excl * (1.0 - a) - cfg.t_eps) / cfg.t_eps, inf)
            pair = torch.stack([m_q, m_a, m_t, m_c], 0)        # [4, chunk, n]
            pair_min, pair_kind = pair.min(0)                 # [chunk, n]
            stop_min = m_t.min(1).values                      # [chunk]
            if extra is not None:  # a pixel-wide decision: it goes with the stop test
                ex = extra[s0:s1]
                stop_min = torch.minimum(stop_min, ex)
                closer = ex[:, None] < pair_min
                pair_kind = torch.where(closer, torch.full_like(pair_kind, 4), pair_kind)
                pair_min = torch.minimum(pair_min, ex[:, None])
            if sel.numel() == 0:
                continue
            pm, pj = pair_min.min(1)                          # per pixel
            pk = pair_kind.gather(1, pj[:, None])[:, 0]
            sl = slice(s0, s1)
            pix[sl], pix_kind[sl], pix_gid[sl] = pm, pk, gid[sel][pj]
            # per Gaussian: its own pair decisions and the stop test of every
            # pixel where it is active or near its support
            touch = near | active
            with_stop = torch.where(touch, torch.minimum(pair_min, stop_min[:, None]), inf)
            if extra is None:
                kind_ws = torch.where(pair_min <= stop_min[:, None], pair_kind, torch.full_like(pair_kind, 2))
            else:
                sk = torch.where(ex < m_t.min(1).values, torch.full_like(ex, 4, dtype=torch.long),
                                 torch.full_like(ex, 2, dtype=torch.long))
                kind_ws = torch.where(pair_min <= stop_min[:, None], pair_kind, sk[:, None].expand_as(pair_kind))
            cm, ci = with_stop.min(0)
            ck = kind_ws.gather(0, ci[None, :])[0]
            better = cm < gm[sel]
            gm[sel] = torch.where(better, cm, gm[sel])
            gk[sel] = torch.where(better, ck, gk[sel])
        gauss = torch.full((N,), float("inf"), dtype=DT)
        gauss_kind = torch.zeros(N, dtype=torch.long)
        if n:
            gauss[gid] = gm[:n]
            gauss_kind[gid] = gk[:n]
    return {"pixel": pix.numpy(), "pixel_kind": pix_kind.numpy(), "pixel_gid": pix_gid.numpy(),
            "gauss": gauss.numpy(), "gauss_kind": gauss_kind.numpy()}


def gaussian_pixel_evals(out: dict) -> int:
    """E_alg: number of (pixel, Gaussian) pairs that were blended."""
    return int(out["n_contrib"].sum())


__all__ = [
    "RasterCfg", "LossCfg", "to_tensors", "quat_to_rotmat", "covariance_3d", "se3_exp", "perturb_pose",
    "project", "composite", "render", "loss_l1", "loss_image_grads", "render_loss", "gradients",
    "weighted_pixel_gradients", "pixel_centers", "gaussian_pixel_evals", "multiview_gradients",
    "multiview_weighted_gradients", "decision_margins", "MARGIN_KINDS", "tile_pixels",
]
