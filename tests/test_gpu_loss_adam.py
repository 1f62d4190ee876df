"""Loss kernel and Adam kernel vs the oracle, on identical inputs."""
import numpy as np
import pytest
import torch

from oracle import adam as oadam
from oracle import render as R
from synth.scene import Camera
from tests._util import compare, ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    ensure_built()
    from paper_2408_12677_gb300.torch_api import Context
    c = Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("H,W", [(48, 64), (70, 100), (680, 1200)])
def test_loss_l1(ctx, H, W):
    from paper_2408_12677_gb300 import abi
    rng = np.random.default_rng(H)
    col = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    dep = rng.uniform(0.5, 4, (H, W)).astype(np.float32)
    trgb = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    tdep = rng.uniform(0.5, 4, (H, W)).astype(np.float32)
    tdep[rng.uniform(0, 1, (H, W)) < 0.1] = 0.0
    trgb[0, 0, :5] = col[0, 0, :5]  # exact zeros of the residual: sign(0) = 0
    t = lambda a: torch.as_tensor(a, device="cuda")
    loss = torch.zeros(1, device="cuda")
    gc = torch.empty((3, H, W), device="cuda")
    gd = torch.empty((H, W), device="cuda")
    cam = abi.make_camera(1, 1, 0, 0, W, H)
    abi.gs_loss_l1(ctx.handle, cam, t(col), t(dep), t(trgb), t(tdep), 0.8, 0.2, loss, gc, gd)
    L, rc, rd = R.loss_image_grads(col, dep, trgb, tdep)
    assert abs(float(loss) - float(L)) <= 1e-5 * abs(float(L))
    np.testing.assert_allclose(gc.cpu().numpy(), rc.numpy(), rtol=1e-6, atol=0)
    np.testing.assert_allclose(gd.cpu().numpy(), rd.numpy(), rtol=1e-6, atol=0)


@pytest.mark.parametrize("n,deg", [(1000, 3), (777, 0), (5, 2)])
def test_adam_matches_oracle_over_steps(ctx, n, deg):
    from paper_2408_12677_gb300 import abi
    # the ABI takes float32 hyper-parameters: give the oracle the same values
    f32 = lambda x: float(np.float32(x))
    cfg = oadam.AdamCfg(lr_means=f32(1e-3), lr_log_scales=f32(5e-3), lr_quats=f32(1e-3), lr_opacity=f32(5e-2),
                        lr_sh_dc=f32(2.5e-3), lr_sh_rest=f32(1.25e-4), beta1=f32(0.9), beta2=f32(0.999),
                        eps=f32(1e-8))
    rng = np.random.default_rng(n)
    size = oadam.flat_size(n, deg)
    p0 = rng.standard_normal(size).astype(np.float32)
    p = torch.tensor(p0, device="cuda")
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    acfg = abi.adam_cfg(lr_means=cfg.lr_means, lr_log_scales=cfg.lr_log_scales, lr_quats=cfg.lr_quats,
                        lr_opacity=cfg.lr_opacity, lr_sh_dc=cfg.lr_sh_dc, lr_sh_rest=cfg.lr_sh_rest, eps=cfg.eps)
    rp, rm, rv = p0.astype(np.float64), np.zeros(size), np.zeros(size)
    lr = oadam.lr_per_element(n, deg, cfg)
    for step in range(1, 6):
        g = (rng.standard_normal(size) * rng.uniform(0.1, 10, size)).astype(np.float32)
        gt = torch.tensor(g, device="cuda")
        # feed the oracle the GPU's own float32 state so each step compares one update
        rp, rm, rv = p.cpu().numpy().astype(np.float64), m.cpu().numpy().astype(np.float64), \
            v.cpu().numpy().astype(np.float64)
        abi.gs_adam_step(ctx.handle, p, gt, m, v, n, deg, acfg, step)
        rp, rm, rv = oadam.adam_step(rp, g, rm, rv, step, lr, cfg)
        torch.cuda.synchronize()
        compare("p", p.cpu().numpy(), rp, 1e-6, 1e-7, 1e-7)
        compare("m", m.cpu().numpy(), rm, 1e-5, 1e-7, 1e-6)
        compare("v", v.cpu().numpy(), rv, 1e-5, 1e-7, 1e-6)
    # zero_grads clears the consumed gradient
    gt = torch.ones(size, device="cuda")
    abi.gs_adam_step(ctx.handle, p, gt, m, v, n, deg, abi.adam_cfg(zero_grads=1), 6)
    torch.cuda.synchronize()
    assert float(gt.abs().max()) == 0.0


@pytest.mark.parametrize("deg,seed", [(0, 1), (3, 2)])
def test_fused_backward_adam_matches_unfused(ctx, deg, seed):
    """gs_render_bwd_adam == gs_render_bwd into zeroed gradients + gs_adam_step,
    over three consecutive iterations (so the moments are non-trivial)."""
    from paper_2408_12677_gb300 import abi
    from paper_2408_12677_gb300.torch_api import GaussianModel, camera_struct
    from synth import workloads
    from synth.scene import Camera, look_at
    cam = Camera(80.0, 75.0, 40.0, 30.0, 84, 60)
    pose = look_at([0.1, 0.2, -0.1], [0.7, 3.0, 0.2])
    P = workloads.random_gaussians(np.random.default_rng(seed), 700, cam, pose, deg, log_scale_range=(-3.5, -1.5),
                                   sh_rest_std=0.15)
    rng = np.random.default_rng(seed + 10)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")
    wc, wd, wa = t(rng.standard_normal((3, 60, 84))), t(rng.standard_normal((60, 84))), t(rng.standard_normal((60, 84)))
    A = GaussianModel(P)
    B = GaussianModel(P)
    camS, view, rcfg = camera_struct(cam), abi.make_viewmat(pose.R, pose.t), abi.raster_cfg()
    acfg = abi.adam_cfg(zero_grads=1)
    for step in range(1, 4):
        pa, pb = torch.zeros(6, device="cuda"), torch.zeros(6, device="cuda")
        abi.gs_render_fwd(ctx.handle, A.gaussians(), camS, view, rcfg)
        abi.gs_render_bwd(ctx.handle, A.gaussians(), camS, view, rcfg, wc, wd, wa, A.grads(), pa)
        abi.gs_adam_step(ctx.handle, A.flat, A.grad, A.m, A.v, A.n, deg, acfg, step)
        abi.gs_render_fwd(ctx.handle, B.gaussians(), camS, view, rcfg)
        abi.gs_render_bwd_adam(ctx.handle, B.gaussians(), camS, view, rcfg, wc, wd, wa, B.flat, B.m, B.v, acfg, step,
                               pb)
        torch.cuda.synchronize()
        for name, x, y in (("p", A.flat, B.flat), ("m", A.m, B.m), ("v", A.v, B.v)):
            xa, ya = x.cpu().numpy(), y.cpu().numpy()
            compare(name, ya, xa, 1e-5, 1e-6 * np.abs(xa).max() + 1e-12, 1e-5)
        # the pose gradient sums every Gaussian's share: a component that cancels
        # carries float32 atomics-order noise of ~1e-6 of the largest component
        pan = pa.cpu().numpy()
        compare("pose", pb.cpu().numpy(), pan, 1e-5, 1e-6 * np.abs(pan).max() + 1e-6, 1e-5)
    assert float(B.grad.abs().max()) == 0.0  # the fused path never touches a gradient buffer


@pytest.mark.parametrize("deg,seed", [(0, 3), (3, 4)])
def test_train_step_matches_three_calls(ctx, deg, seed):
    """gs_train_step (loss in the compositing epilogue, depth scale applied in
    the backward pass) == gs_render_fwd + gs_loss_l1 + gs_render_bwd_adam over
    three iterations: the same loss and the same parameters and moments up to
    float32 atomics order."""
    from paper_2408_12677_gb300 import abi
    from paper_2408_12677_gb300.torch_api import GaussianModel, camera_struct
    from synth import workloads
    from synth.scene import Camera, look_at
    cam = Camera(80.0, 75.0, 40.0, 30.0, 84, 60)
    pose = look_at([0.1, 0.2, -0.1], [0.7, 3.0, 0.2])
    P = workloads.random_gaussians(np.random.default_rng(seed), 700, cam, pose, deg, log_scale_range=(-3.5, -1.5),
                                   sh_rest_std=0.15)
    rng = np.random.default_rng(seed + 10)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")
    trgb = t(rng.uniform(0, 1, (3, 60, 84)))
    tdep_np = rng.uniform(0.5, 4.0, (60, 84))
    tdep_np[:7] = 0.0  # invalid target depth rows
    tdep = t(tdep_np)
    A, B = GaussianModel(P), GaussianModel(P)
    camS, view, rcfg, acfg = camera_struct(cam), abi.make_viewmat(pose.R, pose.t), abi.raster_cfg(), abi.adam_cfg()
    col, dep = torch.empty((3, 60, 84), device="cuda"), torch.empty((60, 84), device="cuda")
    dc, dd = torch.empty_like(col), torch.empty_like(dep)
    la, lb = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
    for step in range(1, 4):
        abi.gs_render_fwd(ctx.handle, A.gaussians(), camS, view, rcfg, col, dep, None)
        abi.gs_loss_l1(ctx.handle, camS, col, dep, trgb, tdep, 0.8, 0.2, la, dc, dd)
        abi.gs_render_bwd_adam(ctx.handle, A.gaussians(), camS, view, rcfg, dc, dd, None, A.flat, A.m, A.v, acfg, step)
        abi.gs_train_step(ctx.handle, B.gaussians(), camS, view, rcfg, trgb, tdep, 0.8, 0.2, lb, B.flat, B.m, B.v,
                          acfg, step)
        torch.cuda.synchronize()
        assert abs(float(la.item()) - float(lb.item())) <= 1e-6 * abs(float(la.item()))
        for name, x, y in (("p", A.flat, B.flat), ("m", A.m, B.m), ("v", A.v, B.v)):
            xa, ya = x.cpu().numpy(), y.cpu().numpy()
            bad = np.abs(xa - ya) > 1e-5 * np.abs(xa) + 1e-6 * np.abs(xa).max() + 1e-12
            assert bad.sum() <= max(2, int(1e-4 * xa.size)), (name, step, int(bad.sum()))


def test_train_step_device_step_and_empty_map(ctx):
    """gs_train_step with step = 0 takes the Adam step from the context's
    device counter, which the projection advances once per call: three such
    calls from counter 0 give the parameters, moments and losses of explicit
    steps 1, 2, 3.  With no Gaussians the loss is still reduced (of the
    background image) and the counter still advances."""
    from paper_2408_12677_gb300 import abi
    from paper_2408_12677_gb300.torch_api import GaussianModel, camera_struct
    from synth import workloads
    from synth.scene import Camera, look_at
    cam = Camera(80.0, 75.0, 40.0, 30.0, 84, 60)
    pose = look_at([0.1, 0.2, -0.1], [0.7, 3.0, 0.2])
    P = workloads.random_gaussians(np.random.default_rng(8), 600, cam, pose, 1, log_scale_range=(-3.5, -1.5),
                                   sh_rest_std=0.15)
    rng = np.random.default_rng(9)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")
    trgb = t(rng.uniform(0, 1, (3, 60, 84)))
    tdep = t(rng.uniform(0.5, 4.0, (60, 84)))
    A, B = GaussianModel(P), GaussianModel(P)
    camS, view, rcfg, acfg = camera_struct(cam), abi.make_viewmat(pose.R, pose.t), abi.raster_cfg(), abi.adam_cfg()
    la, lb = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
    abi.gs_ctx_set_adam_step(ctx.handle, 0)
    for step in range(1, 4):
        abi.gs_train_step(ctx.handle, A.gaussians(), camS, view, rcfg, trgb, tdep, 0.8, 0.2, la, A.flat, A.m, A.v,
                          acfg, step)
        abi.gs_train_step(ctx.handle, B.gaussians(), camS, view, rcfg, trgb, tdep, 0.8, 0.2, lb, B.flat, B.m, B.v,
                          acfg, 0)
        torch.cuda.synchronize()
        assert abs(float(la.item()) - float(lb.item())) <= 1e-6 * abs(float(la.item()))
        for name, x, y in (("p", A.flat, B.flat), ("m", A.m, B.m), ("v", A.v, B.v)):
            xa, ya = x.cpu().numpy(), y.cpu().numpy()
            bad = np.abs(xa - ya) > 1e-5 * np.abs(xa) + 1e-6 * np.abs(xa).max() + 1e-12
            assert bad.sum() <= max(2, int(1e-4 * xa.size)), (name, step, int(bad.sum()))
    # an empty map: the loss of the background image, and the counter moves on to 4
    empty = {"means": np.zeros((0, 3), np.float32), "log_scales": np.zeros((0, 3), np.float32),
             "quats": np.zeros((0, 4), np.float32), "opacity_logits": np.zeros(0, np.float32),
             "sh": np.zeros((0, 4, 3), np.float32), "sh_degree": 1}
    E = GaussianModel(empty)
    le = torch.full((1,), -1.0, device="cuda")
    abi.gs_train_step(ctx.handle, E.gaussians(), camS, view, abi.raster_cfg(bg=(0.25, 0.5, 0.75)), trgb, tdep, 0.8,
                      0.2, le, E.flat, E.m, E.v, acfg, 0)
    torch.cuda.synchronize()
    bg = np.array([0.25, 0.5, 0.75], np.float64)[:, None, None]
    want = 0.8 * np.abs(bg - trgb.cpu().numpy().astype(np.float64)).mean() + \
        0.2 * np.abs(tdep.cpu().numpy().astype(np.float64)).mean()  # rendered depth 0, every target valid
    assert abs(float(le.item()) - want) <= 1e-5 * want
    # the fourth device step: one more step = 0 call equals explicit step 5 after a step-4 call
    abi.gs_train_step(ctx.handle, A.gaussians(), camS, view, rcfg, trgb, tdep, 0.8, 0.2, la, A.flat, A.m, A.v,
                      acfg, 5)
    abi.gs_train_step(ctx.handle, B.gaussians(), camS, view, rcfg, trgb, tdep, 0.8, 0.2, lb, B.flat, B.m, B.v,
                      acfg, 0)
    torch.cuda.synchronize()
    xa, ya = A.flat.cpu().numpy(), B.flat.cpu().numpy()
    bad = np.abs(xa - ya) > 1e-5 * np.abs(xa) + 1e-6 * np.abs(xa).max() + 1e-12
    assert bad.sum() <= max(2, int(1e-4 * xa.size))
