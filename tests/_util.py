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
        if not os.path.exists(abi.LIB_PATH):
            build.build()
    return abi.load()


def compare(name, got, ref, rtol, atol, norm_rtol, flip_budget=0, report=None):
    """Element-wise |got - ref| <= rtol |ref| + atol except for at most
    ``flip_budget`` elements, and ||got - ref|| / ||ref|| <= norm_rtol."""
    got = np.asarray(got, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    assert got.shape == ref.shape, (name, got.shape, ref.shape)
    assert np.isfinite(got).all(), f"{name}: non-finite values"
    err = np.abs(got - ref)
    bad = err > rtol * np.abs(ref) + atol
    nref = np.linalg.norm(ref)
    nrel = np.linalg.norm(got - ref) / nref if nref > 0 else np.linalg.norm(got - ref)
    info = {"name": name, "n": int(ref.size), "bad": int(bad.sum()), "max_err": float(err.max(initial=0.0)),
            "norm_rel": float(nrel)}
    if report is not None:
        report.append(info)
    assert int(bad.sum()) <= flip_budget, f"{name}: {info} (budget {flip_budget}); worst idx {np.argsort(-err)[:5]}"
    assert nrel <= norm_rtol, f"{name}: {info} (norm tolerance {norm_rtol})"
    return info


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
