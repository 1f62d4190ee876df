"""Runs a fixed set of calls through one build of the library and saves what
they return, for tests/test_gpu_checked.py.

usage: python -m tests._checked_run {normal|checked} OUT.npz

The cases: a small map (forward images, L1 loss, backward gradients, two
fused training steps), a ragged 333 x 77 image, two views in one batched
forward + backward, and tile lists longer than the per-tile sort holds (the
radix binning).  Then the bounds report: gs_sync_status must find nothing,
and a bounds fault set from the host must come back as GS_ERR_BOUNDS once."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    which, out_path = sys.argv[1], sys.argv[2]
    import torch

    from paper_2408_12677_gb300 import abi
    abi.load(abi.CHECKED_LIB_PATH if which == "checked" else abi.LIB_PATH)
    from paper_2408_12677_gb300.torch_api import Context, GaussianModel, camera_struct
    from synth import workloads
    from synth.scene import Camera, look_at

    ctx = Context(0)
    h = ctx.handle
    out = {"checked": np.array(abi.gs_bounds_checked())}
    dev = "cuda"
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=dev)
    rcfg, acfg = abi.raster_cfg(), abi.adam_cfg(zero_grads=1)

    def render(model, cam, view, tag):
        W, H = cam.width, cam.height
        col, dep, alp = (torch.zeros((3, H, W), device=dev), torch.zeros((H, W), device=dev),
                         torch.zeros((H, W), device=dev))
        abi.gs_render_fwd(h, model.gaussians(), camera_struct(cam), view, rcfg, col, dep, alp)
        out[tag + "_color"], out[tag + "_depth"], out[tag + "_alpha"] = (x.cpu().numpy() for x in (col, dep, alp))
        return col, dep

    # a small map: forward, loss, backward, then two fused training steps
    w = workloads.tiny_random(seed=71, n=600, sh_degree=3, sh_rest_std=0.1)
    v = w.views[0]
    view = abi.make_viewmat(v.pose.R, v.pose.t)
    model = GaussianModel(w.params)
    col, dep = render(model, v.cam, view, "small")
    trgb, tdep = t(v.target_rgb), t(v.target_depth)
    loss = torch.zeros(1, device=dev)
    dc, dd = torch.empty_like(col), torch.empty_like(dep)
    abi.gs_loss_l1(h, camera_struct(v.cam), col, dep, trgb, tdep, 0.8, 0.2, loss, dc, dd)
    model.grad.zero_()
    abi.gs_render_bwd(h, model.gaussians(), camera_struct(v.cam), view, rcfg, dc, dd, None, model.grads())
    out["small_loss"] = loss.cpu().numpy()
    out["small_grad"] = model.grad.cpu().numpy()
    for step in (1, 2):
        abi.gs_train_step(h, model.gaussians(), camera_struct(v.cam), view, rcfg, trgb, tdep, 0.8, 0.2, loss,
                          model.flat, model.m, model.v, acfg, step)
    out["small_params"] = model.flat.cpu().numpy()

    # a ragged image (partial tiles on both edges)
    cam = Camera(150.0, 150.0, 166.5, 38.5, 333, 77)
    pose = look_at([0.0, 0.0, 0.0], [0.0, 0.0, 3.0])
    P = workloads.random_gaussians(np.random.default_rng(72), 3000, cam, pose, 1, sh_rest_std=0.1)
    render(GaussianModel(P), cam, abi.make_viewmat(pose.R, pose.t), "ragged")

    # two views in one batched forward + backward
    cams = [Camera(80.0, 75.0, 40.0, 30.0, 84, 60), Camera(70.0, 70.0, 33.0, 27.0, 66, 52)]
    poses = [look_at([0.1, 0.2, -0.1], [0.7, 3.0, 0.2]), look_at([0.3, 0.1, -0.2], [0.6, 3.1, 0.1])]
    P = workloads.random_gaussians(np.random.default_rng(73), 1500, cams[0], poses[0], 3, sh_rest_std=0.1)
    mb = GaussianModel(P)
    cs, vms = [camera_struct(c) for c in cams], [abi.make_viewmat(p.R, p.t) for p in poses]
    cols = [torch.zeros((3, c.height, c.width), device=dev) for c in cams]
    deps = [torch.zeros((c.height, c.width), device=dev) for c in cams]
    abi.gs_render_fwd_batched(h, mb.gaussians(), cs, vms, rcfg, cols, deps, None)
    for k in range(2):
        out[f"batched_color{k}"] = cols[k].cpu().numpy()
    rng = np.random.default_rng(74)
    wc = [t(rng.standard_normal((3, c.height, c.width)) * 1e-3) for c in cams]
    wd = [t(rng.standard_normal((c.height, c.width)) * 1e-3) for c in cams]
    mb.grad.zero_()
    abi.gs_render_bwd_batched(h, mb.gaussians(), cs, vms, rcfg, wc, wd, None, mb.grads())
    out["batched_grad"] = mb.grad.cpu().numpy()

    # tile lists longer than the per-tile sort holds: the radix binning
    cam = Camera(60.0, 60.0, 32.0, 24.0, 64, 48)
    pose = look_at([0.0, 0.0, 0.0], [0.0, 0.0, 3.0])
    P = workloads.random_gaussians(np.random.default_rng(75), 6000, cam, pose, 0, log_scale_range=(0.0, 0.5))
    render(GaussianModel(P), cam, abi.make_viewmat(pose.R, pose.t), "long")

    torch.cuda.synchronize()
    abi.gs_sync_status(h)  # raises on GS_ERR_BOUNDS
    out["bounds_clean"] = np.array(True)
    abi.gs_ctx_inject_bounds_fault(h)
    try:
        abi.gs_sync_status(h)
        out["injected_reported"] = np.array(False)
    except RuntimeError as e:
        out["injected_reported"] = np.array("GS_ERR_BOUNDS" in str(e))
    abi.gs_sync_status(h)  # cleared
    np.savez(out_path, **out)


if __name__ == "__main__":
    main()
