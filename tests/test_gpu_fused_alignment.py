"""The fused projection backward + Adam stages each block's slices of the
parameter and moment buffers in shared memory and writes them back.  The
update must not depend on where the slices fall: map sizes N = 1, 2, 3
(mod 4) put the five slices of a block at different offsets within their
16-byte chunks, and the buffers themselves start 0-3 floats past a 16-byte
boundary.  Reference: the unfused path (gradients into zeroed buffers, then
gs_adam_step) on 16-byte aligned buffers."""
import numpy as np
import pytest
import torch

from tests._util import compare, ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    ensure_built()
    from paper_2408_12677_gb300.torch_api import Context
    c = Context(0)
    yield c
    c.close()


def _shifted(model, offsets):
    """Moves the model's parameter and moment buffers to storage that starts
    offsets = (params, m, v) floats past a 16-byte boundary."""
    from paper_2408_12677_gb300.torch_api import _views
    outs = []
    for src, o in zip((model.flat, model.m, model.v), offsets):
        big = torch.zeros(src.numel() + 8, device=src.device)
        assert big.data_ptr() % 16 == 0
        dst = big[o:o + src.numel()]
        dst.copy_(src)
        assert dst.data_ptr() % 16 == 4 * o
        outs.append(dst)
    model.flat, model.m, model.v = outs
    model.p = _views(model.flat, model.n, model.sh_degree)


@pytest.mark.parametrize("n,deg,offsets", [(701, 3, (1, 2, 3)), (702, 3, (3, 0, 1)), (703, 1, (2, 3, 0)),
                                           (705, 2, (0, 1, 2)), (33, 3, (3, 3, 3)), (5, 0, (1, 0, 2))])
def test_fused_adam_any_alignment(ctx, n, deg, offsets):
    from paper_2408_12677_gb300 import abi
    from paper_2408_12677_gb300.torch_api import GaussianModel, camera_struct
    from synth import workloads
    from synth.scene import Camera, look_at
    cam = Camera(80.0, 75.0, 40.0, 30.0, 84, 60)
    pose = look_at([0.1, 0.2, -0.1], [0.7, 3.0, 0.2])
    P = workloads.random_gaussians(np.random.default_rng(n), n, cam, pose, deg, log_scale_range=(-3.0, -1.5),
                                   sh_rest_std=0.15)
    rng = np.random.default_rng(n + 1)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")
    wc, wd = t(rng.standard_normal((3, 60, 84))), t(rng.standard_normal((60, 84)))
    A, B = GaussianModel(P), GaussianModel(P)
    for mdl in (A, B):
        mdl.m.copy_(torch.as_tensor(rng.normal(0, 1e-4, mdl.m.numel()), dtype=torch.float32))
        mdl.v.copy_(torch.as_tensor(rng.uniform(0, 1e-6, mdl.v.numel()), dtype=torch.float32))
    B.m.copy_(A.m)
    B.v.copy_(A.v)
    _shifted(B, offsets)
    camS, view, rcfg = camera_struct(cam), abi.make_viewmat(pose.R, pose.t), abi.raster_cfg()
    acfg = abi.adam_cfg(zero_grads=1)
    for step in range(1, 4):
        abi.gs_render_fwd(ctx.handle, A.gaussians(), camS, view, rcfg)
        abi.gs_render_bwd(ctx.handle, A.gaussians(), camS, view, rcfg, wc, wd, None, A.grads())
        abi.gs_adam_step(ctx.handle, A.flat, A.grad, A.m, A.v, A.n, deg, acfg, step)
        abi.gs_render_fwd(ctx.handle, B.gaussians(), camS, view, rcfg)
        abi.gs_render_bwd_adam(ctx.handle, B.gaussians(), camS, view, rcfg, wc, wd, None, B.flat, B.m, B.v, acfg,
                               step)
        torch.cuda.synchronize()
        for name, x, y in (("p", A.flat, B.flat), ("m", A.m, B.m), ("v", A.v, B.v)):
            xa, ya = x.cpu().numpy(), y.cpu().numpy()
            compare(f"{name} step {step}", ya, xa, 1e-5, 1e-6 * np.abs(xa).max() + 1e-12, 1e-5)


@pytest.mark.parametrize("offsets", [(1, 2, 3), (2, 3, 1)])
def test_batched_fused_adam_any_alignment(ctx, offsets):
    """The multi-view fused kernel (gradients of three views summed before the
    one Adam update) on shifted buffers of a map with N = 3 (mod 4)."""
    from paper_2408_12677_gb300 import abi
    from paper_2408_12677_gb300.torch_api import GaussianModel, camera_struct
    from synth import workloads
    from synth.scene import Camera, look_at
    n, deg = 1203, 3
    cams_py = [Camera(80.0, 75.0, 40.0, 30.0, 84, 60), Camera(70.0, 70.0, 33.0, 27.0, 66, 52),
               Camera(90.0, 88.0, 45.0, 31.0, 90, 64)]
    poses = [look_at([0.1, 0.2, -0.1], [0.7, 3.0, 0.2]), look_at([0.3, 0.1, -0.2], [0.6, 3.1, 0.1]),
             look_at([-0.1, 0.25, -0.1], [0.8, 2.9, 0.3])]
    P = workloads.random_gaussians(np.random.default_rng(7), n, cams_py[0], poses[0], deg,
                                   log_scale_range=(-3.0, -1.5), sh_rest_std=0.15)
    rng = np.random.default_rng(8)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")
    wc = [t(rng.standard_normal((3, c.height, c.width)) * 1e-3) for c in cams_py]
    wd = [t(rng.standard_normal((c.height, c.width)) * 1e-3) for c in cams_py]
    cams = [camera_struct(c) for c in cams_py]
    vms = [abi.make_viewmat(p.R, p.t) for p in poses]
    rcfg, acfg = abi.raster_cfg(), abi.adam_cfg(zero_grads=1)
    A, B = GaussianModel(P), GaussianModel(P)
    A.m.normal_(0, 1e-4)
    A.v.uniform_(0, 1e-6)
    B.m.copy_(A.m)
    B.v.copy_(A.v)
    _shifted(B, offsets)
    for step in (1, 2):
        abi.gs_render_fwd_batched(ctx.handle, A.gaussians(), cams, vms, rcfg)
        abi.gs_render_bwd_batched(ctx.handle, A.gaussians(), cams, vms, rcfg, wc, wd, None, A.grads())
        abi.gs_adam_step(ctx.handle, A.flat, A.grad, A.m, A.v, A.n, deg, acfg, step)
        abi.gs_render_fwd_batched(ctx.handle, B.gaussians(), cams, vms, rcfg)
        abi.gs_render_bwd_adam_batched(ctx.handle, B.gaussians(), cams, vms, rcfg, wc, wd, None, B.flat, B.m, B.v,
                                       acfg, step)
        torch.cuda.synchronize()
        for name, x, y in (("params", A.flat, B.flat), ("m", A.m, B.m), ("v", A.v, B.v)):
            xa, ya = x.cpu().numpy(), y.cpu().numpy()
            # float32 atomics order: a near-zero gradient can flip Adam's step sign
            bad = np.abs(xa - ya) > 1e-5 * np.abs(xa) + 1e-7 * max(np.abs(xa).max(), 1e-30)
            assert bad.sum() <= max(4, int(1e-4 * xa.size)), (name, step, int(bad.sum()))
