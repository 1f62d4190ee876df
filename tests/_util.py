"""Shared helpers for the parity tests (comparison with tolerance budgets,
building the library once, moving synthetic workloads to the GPU)."""
from __future__ import annotations

import os
import threading

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_lock = threading.Lock()


def ensure_built():
    from paper_2408_12677_gb300 import abi, build
    with _lock:
        if not (os.path.exists(abi.LIB_PATH) and os.path.exists(abi.CHECKED_LIB_PATH)):
            build.build()
    return abi.load()


MARGIN_KINDS = ("q = 9", "alpha = 1/255", "T (1 - alpha) = 1e-4", "alpha = 0.99", "L1 residual = 0")
FLIP_EPS = 1e-4  # relative distance to a threshold within which float32 may decide the other way


def compare(name, got, ref, rtol, atol, norm_rtol, flip_budget=0, report=None, margins=None, kinds=None,
            flip_eps=FLIP_EPS, groups=None):
    """Element-wise |got - ref| <= rtol |ref| + atol except for at most
    ``flip_budget`` elements ("flips"), and ||got - ref|| / ||ref|| <= norm_rtol.
    With ``groups`` (one id per element) the budget counts distinct groups
    among the flips instead of elements: one flipped decision of a Gaussian
    moves all of that Gaussian's gradient elements.

    With ``margins`` (one per element: the oracle's relative
    float64 distance of the decisions behind the element to their thresholds,
    ``kinds`` naming the nearest one), every element beyond the tolerance must
    lie within ``flip_eps`` of a threshold -- a float32 / float64 decision
    flip -- and each is listed in the report with its threshold and distance;
    an element beyond the tolerance away from every threshold fails."""
    got = np.asarray(got, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    assert got.shape == ref.shape, (name, got.shape, ref.shape)
    assert np.isfinite(got).all(), f"{name}: non-finite values"
    err = np.abs(got - ref)
    tol = rtol * np.abs(ref) + atol
    bad = err > tol
    nref = np.linalg.norm(ref)
    nrel = np.linalg.norm(got - ref) / nref if nref > 0 else np.linalg.norm(got - ref)
    info = {"name": name, "n": int(ref.size), "bad": int(bad.sum()), "max_err": float(err.max(initial=0.0)),
            "norm_rel": float(nrel), "budget": int(flip_budget), "flips": []}
    unexplained = []
    if bad.any():
        idx = np.nonzero(bad)[0]
        if margins is not None:
            mg = np.asarray(margins, np.float64).ravel()
            kd = None if kinds is None else np.asarray(kinds).ravel()
            assert mg.size == ref.size and (kd is None or kd.size == ref.size), (name, mg.size, ref.size)
            for i in idx.tolist():
                rec = {"i": i, "got": float(got[i]), "ref": float(ref[i]), "err": float(err[i]),
                       "tol": float(tol[i]), "margin": float(mg[i]),
                       "kind": MARGIN_KINDS[int(kd[i])] if kd is not None else None}
                info["flips"].append(rec)
                if not mg[i] <= flip_eps:
                    unexplained.append(rec)
        else:
            info["flips"] = [{"i": int(i), "got": float(got[i]), "ref": float(ref[i]), "err": float(err[i]),
                              "tol": float(tol[i])} for i in idx.tolist()]
    if report is not None:
        report.append(info)
    assert not unexplained, f"{name}: {len(unexplained)} elements beyond tolerance away from every threshold: " \
                            f"{unexplained[:5]}"
    n_flips = int(bad.sum()) if groups is None else int(np.unique(np.asarray(groups).ravel()[bad]).size)
    info["flipped_groups"] = None if groups is None else n_flips
    assert n_flips <= flip_budget, f"{name}: {info['bad']} flips (budget {flip_budget}): {info['flips'][:5]}"
    assert nrel <= norm_rtol, f"{name}: norm rel {nrel:.3e} (tolerance {norm_rtol})"
    return info


def residual_margins(color, depth, target_rgb, target_depth):
    """Per pixel, the relative distance of the L1 loss residuals (Eq. 12 plus
    the depth term) to 0, where their sign -- the image gradient -- flips:
    min over the channels (and the depth where its target is valid) of
    |r| / (|value| + 0.01); within 1e-4 the float32 render (image tolerance
    1e-4 |value| + 1e-6) may give the other sign."""
    c = np.asarray(color, np.float64).reshape(3, -1)
    tc = np.asarray(target_rgb, np.float64).reshape(3, -1)
    d = np.asarray(depth, np.float64).reshape(-1)
    td = np.asarray(target_depth, np.float64).reshape(-1)
    m = (np.abs(c - tc) / (np.abs(c) + 0.01)).min(0)
    md = np.where(td > 0, np.abs(d - td) / (np.abs(d) + 0.01), np.inf)
    return np.minimum(m, md)


def margins_over_views(params, deg, cams, poses, extras=None):
    """Per-Gaussian decision margins (``R.decision_margins``) of several views
    of one map: the smallest over the views (``extras``: per view a further
    per-pixel margin, e.g. ``residual_margins``)."""
    from oracle import render as R
    out = None
    for v, (cam, (Rm, t)) in enumerate(zip(cams, poses)):
        m = R.decision_margins(params, deg, cam, np.asarray(Rm, np.float64), np.asarray(t, np.float64),
                               pixel_extra=None if extras is None else extras[v])
        if out is None:
            out = {"gauss": m["gauss"].copy(), "gauss_kind": m["gauss_kind"].copy()}
        else:
            better = m["gauss"] < out["gauss"]
            out["gauss"][better] = m["gauss"][better]
            out["gauss_kind"][better] = m["gauss_kind"][better]
    return out


def to_gpu_model(params):
    from paper_2408_12677_gb300.torch_api import GaussianModel
    return GaussianModel(params)


def oracle_params(params):
    from oracle import render as R
    return R.to_tensors({k: np.asarray(params[k], np.float64) for k in R.PARAM_NAMES})


def gpu_render(ctx, model, cam, pose, **cfg):
    """Run gs_render_fwd; returns numpy colour, depth, alpha."""
    import torch
    from paper_2408_12677_gb300 import abi
    from paper_2408_12677_gb300.torch_api import camera_struct
    H, W = cam.height, cam.width
    color = torch.empty((3, H, W), device="cuda")
    depth = torch.empty((H, W), device="cuda")
    alpha = torch.empty((H, W), device="cuda")
    abi.gs_render_fwd(ctx.handle, model.gaussians(), camera_struct(cam), abi.make_viewmat(pose.R, pose.t),
                      abi.raster_cfg(**cfg), color, depth, alpha)
    torch.cuda.synchronize()
    return color.cpu().numpy(), depth.cpu().numpy(), alpha.cpu().numpy()


def gpu_backward(ctx, model, cam, pose, wc, wd, wa, **cfg):
    """gs_render_bwd of the last forward with upstream images (numpy); returns
    numpy gradients per parameter array and the pose twist gradient."""
    import torch
    from paper_2408_12677_gb300 import abi
    from paper_2408_12677_gb300.torch_api import camera_struct
    model.grad.zero_()
    gp = torch.zeros(6, device="cuda")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")
    abi.gs_render_bwd(ctx.handle, model.gaussians(), camera_struct(cam), abi.make_viewmat(pose.R, pose.t),
                      abi.raster_cfg(**cfg), t(wc), t(wd), None if wa is None else t(wa), model.grads(), gp)
    torch.cuda.synchronize()
    out = {k: v.detach().cpu().numpy().copy() for k, v in model.g.items()}
    out["pose"] = gp.cpu().numpy()
    return out
