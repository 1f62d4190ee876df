"""Batched multi-view form on the GPU: several views of uneven resolution
rendered, scored and differentiated against one map in single launches.

Checked against (i) the FP64 oracle per view (images) and its multi-view
objective (gradients summed over the views, per-view pose gradients), with
the tolerances of the single-view tests, and (ii) the single-view entry
points run one view at a time: the batched forward images must be bit-for-bit
those of the single-view calls (same arithmetic, same per-tile order), the
summed gradients and the Adam step equal up to float32 atomics order."""
import numpy as np
import pytest
import torch

from oracle import render as R
from synth import workloads
from synth.scene import Camera, look_at
from tests._util import compare, ensure_built, margins_over_views, oracle_params, to_gpu_model
from tests.test_gpu_grad import check_grad_arrays

pytestmark = pytest.mark.gpu

NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


@pytest.fixture(scope="module")
def ctx():
    ensure_built()
    from paper_2408_12677_gb300.torch_api import Context
    c = Context(0)
    yield c
    c.close()


def _structs(views):
    from paper_2408_12677_gb300 import abi
    from paper_2408_12677_gb300.torch_api import camera_struct
    return [camera_struct(v.cam) for v in views], [abi.make_viewmat(v.pose.R, v.pose.t) for v in views]


def _batched_render(ctx, model, views, **cfg):
    from paper_2408_12677_gb300 import abi
    cams, vms = _structs(views)
    col = [torch.empty((3, v.cam.height, v.cam.width), device="cuda") for v in views]
    dep = [torch.empty((v.cam.height, v.cam.width), device="cuda") for v in views]
    alp = [torch.empty((v.cam.height, v.cam.width), device="cuda") for v in views]
    abi.gs_render_fwd_batched(ctx.handle, model.gaussians(), cams, vms, abi.raster_cfg(**cfg), col, dep, alp)
    torch.cuda.synchronize()
    return [(c.cpu().numpy(), d.cpu().numpy(), a.cpu().numpy()) for c, d, a in zip(col, dep, alp)]


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")


def _batched_backward(ctx, model, views, wc, wd, wa, **cfg):
    from paper_2408_12677_gb300 import abi
    cams, vms = _structs(views)
    model.grad.zero_()
    gp = torch.zeros((len(views), 6), device="cuda")
    abi.gs_render_bwd_batched(ctx.handle, model.gaussians(), cams, vms, abi.raster_cfg(**cfg),
                              [_t(x) for x in wc], [_t(x) for x in wd],
                              None if wa is None else [_t(x) for x in wa], model.grads(), gp)
    torch.cuda.synchronize()
    out = {k: v.detach().cpu().numpy().copy() for k, v in model.g.items()}
    out["pose"] = gp.cpu().numpy()
    return out


def _flip_budget(npx):
    return max(1, int(1e-5 * npx))


@pytest.mark.parametrize("tile", [(16, 16), (8, 32), (32, 8)])
def test_batched_forward_matches_oracle(ctx, tile):
    w = workloads.tiny_multi_view(n=500)
    model = to_gpu_model(w.params)
    imgs = _batched_render(ctx, model, w.views, tile_w=tile[0], tile_h=tile[1])
    P = oracle_params(w.params)
    for v, (col, dep, alp) in zip(w.views, imgs):
        R64, t64 = v.pose.R.astype(np.float64), v.pose.t.astype(np.float64)
        o = R.render(P, 0, v.cam, R64, t64, prefilter=True)
        mg = R.decision_margins(w.params, 0, v.cam, R64, t64)
        mk = dict(margins=mg["pixel"], kinds=mg["pixel_kind"])
        npx = v.cam.width * v.cam.height
        assert np.count_nonzero(o["alpha"].numpy() > 0.05) > npx // 4  # the cloud is in view
        for c in range(3):
            compare(f"color{c}", col[c], o["color"][c].numpy(), 1e-4, 1e-6, 1e-4, _flip_budget(npx), **mk)
        compare("depth", dep, o["depth"].numpy(), 1e-4, 1e-6, 1e-4, _flip_budget(npx), **mk)
        compare("alpha", alp, o["alpha"].numpy(), 1e-4, 1e-6, 1e-4, _flip_budget(npx), **mk)


@pytest.mark.parametrize("deg,tile", [(0, (16, 16)), (3, (8, 32))])
def test_batched_backward_matches_oracle(ctx, deg, tile):
    w = workloads.tiny_multi_view(seed=1006, n=400, sh_degree=deg, sh_rest_std=0.15 if deg else 0.0)
    rng = np.random.default_rng(31 + deg)
    wc = [rng.standard_normal((3, v.cam.height, v.cam.width)).astype(np.float32) for v in w.views]
    wd = [rng.standard_normal((v.cam.height, v.cam.width)).astype(np.float32) for v in w.views]
    wa = [rng.standard_normal((v.cam.height, v.cam.width)).astype(np.float32) for v in w.views]
    model = to_gpu_model(w.params)
    _batched_render(ctx, model, w.views, tile_w=tile[0], tile_h=tile[1])
    g = _batched_backward(ctx, model, w.views, wc, wd, wa, tile_w=tile[0], tile_h=tile[1])
    poses = [(v.pose.R.astype(np.float64), v.pose.t.astype(np.float64)) for v in w.views]
    og = R.multiview_weighted_gradients(w.params, deg, [v.cam for v in w.views], poses,
                                        [x.astype(np.float64) for x in wc], [x.astype(np.float64) for x in wd],
                                        [x.astype(np.float64) for x in wa])
    check_grad_arrays(g, og, margins_over_views(w.params, deg, [v.cam for v in w.views], poses))


def _mid_views(n_views=3):
    sizes = ((160, 120, 150.0), (96, 64, 90.0), (200, 152, 190.0), (48, 40, 45.0))
    eyes = ([0.0, 0.0, 0.0], [0.3, -0.3, 0.1], [-0.25, 0.3, -0.15], [0.1, 0.2, 0.3])
    views = []
    rng = np.random.default_rng(5)
    for k in range(n_views):
        wdt, hgt, f = sizes[k]
        cam = Camera(f, f, wdt / 2.0, hgt / 2.0, wdt, hgt)
        pose = look_at(eyes[k], [2.5, 0.0, 0.0])
        views.append(workloads.View(cam, pose, rng.uniform(0, 1, (3, hgt, wdt)).astype(np.float32),
                                    rng.uniform(0.5, 4.0, (hgt, wdt)).astype(np.float32)))
    P = workloads.random_gaussians(rng, 20000, views[0].cam, views[0].pose, 3, z_range=(1.5, 3.5),
                                   log_scale_range=(-4.5, -2.0), sh_rest_std=0.1)
    return P, views


def _single_render(ctx, model, v, **cfg):
    from tests._util import gpu_render
    return gpu_render(ctx, model, v.cam, v.pose, **cfg)


def test_batched_forward_is_bitwise_single_view(ctx):
    P, views = _mid_views(4)
    model = to_gpu_model(P)
    imgs = _batched_render(ctx, model, views)
    for v, (col, dep, alp) in zip(views, imgs):
        c1, d1, a1 = _single_render(ctx, model, v)
        assert np.array_equal(col, c1) and np.array_equal(dep, d1) and np.array_equal(alp, a1)


def test_batched_backward_equals_sum_of_single_views(ctx):
    from tests._util import gpu_backward
    P, views = _mid_views(3)
    rng = np.random.default_rng(9)
    wc = [rng.standard_normal((3, v.cam.height, v.cam.width)).astype(np.float32) for v in views]
    wd = [rng.standard_normal((v.cam.height, v.cam.width)).astype(np.float32) for v in views]
    model = to_gpu_model(P)
    _batched_render(ctx, model, views)
    gb = _batched_backward(ctx, model, views, wc, wd, None)
    total = None
    poses = []
    for v, c, d in zip(views, wc, wd):
        _single_render(ctx, model, v)
        g = gpu_backward(ctx, model, v.cam, v.pose, c, d, None)
        poses.append(g.pop("pose"))
        total = g if total is None else {k: total[k] + g[k] for k in total}
    for k in NAMES:
        compare(k, gb[k], total[k], 1e-3, 1e-6 * np.abs(total[k]).max(), 1e-5, max(2, int(1e-3 * total[k].size)))
    compare("pose", gb["pose"], np.stack(poses), 1e-3, 1e-6 * np.abs(np.stack(poses)).max(), 1e-5)


def test_batched_loss_is_sum_of_view_losses(ctx):
    from paper_2408_12677_gb300 import abi
    P, views = _mid_views(3)
    model = to_gpu_model(P)
    cams, vms = _structs(views)
    col = [torch.rand((3, v.cam.height, v.cam.width), device="cuda") for v in views]
    dep = [torch.rand((v.cam.height, v.cam.width), device="cuda") * 4 for v in views]
    trgb = [_t(v.target_rgb) for v in views]
    tdep = [_t(v.target_depth) for v in views]
    tdep[1][:5] = 0.0  # invalid depth rows are excluded from the depth term
    loss = torch.zeros(1, device="cuda")
    dLdc = [torch.empty_like(c) for c in col]
    dLdd = [torch.empty_like(d) for d in dep]
    abi.gs_loss_l1_batched(ctx.handle, cams, col, dep, trgb, tdep, 0.8, 0.2, loss, dLdc, dLdd)
    total = 0.0
    for v in range(len(views)):
        l1 = torch.zeros(1, device="cuda")
        gc = torch.empty_like(col[v])
        gd = torch.empty_like(dep[v])
        abi.gs_loss_l1(ctx.handle, cams[v], col[v], dep[v], trgb[v], tdep[v], 0.8, 0.2, l1, gc, gd)
        torch.cuda.synchronize()
        total += float(l1.item())
        assert torch.equal(gc, dLdc[v]) and torch.equal(gd, dLdd[v])
        _, ogc, ogd = R.loss_image_grads(col[v].double().cpu(), dep[v].double().cpu(), views[v].target_rgb,
                                         tdep[v].cpu().numpy())
        assert np.allclose(gc.cpu().numpy(), ogc.numpy(), rtol=1e-6, atol=1e-12)
        assert np.allclose(gd.cpu().numpy(), ogd.numpy(), rtol=1e-6, atol=1e-12)
    assert abs(float(loss.item()) - total) <= 1e-6 * abs(total)


@pytest.mark.parametrize("deg", [0, 3])
def test_batched_fused_adam_equals_unfused(ctx, deg):
    """gs_render_bwd_adam_batched == gs_render_bwd_batched into zeroed
    gradients followed by gs_adam_step (the multi-view fused kernel)."""
    from paper_2408_12677_gb300 import abi
    P, views = _mid_views(3)
    if deg == 0:
        P = dict(P, sh=np.ascontiguousarray(P["sh"][:, :1, :]), sh_degree=0)
    rng = np.random.default_rng(13)
    wc = [_t(rng.standard_normal((3, v.cam.height, v.cam.width)) * 1e-3) for v in views]
    wd = [_t(rng.standard_normal((v.cam.height, v.cam.width)) * 1e-3) for v in views]
    cams, vms = _structs(views)
    acfg = abi.adam_cfg(zero_grads=1)
    rcfg = abi.raster_cfg()
    ma, mb = to_gpu_model(P), to_gpu_model(P)
    for mdl in (ma, mb):
        mdl.m.normal_(0, 1e-4)
        mdl.v.uniform_(0, 1e-6)
    mb.m.copy_(ma.m)
    mb.v.copy_(ma.v)
    for step in (1, 2):
        abi.gs_render_fwd_batched(ctx.handle, ma.gaussians(), cams, vms, rcfg)
        abi.gs_render_bwd_adam_batched(ctx.handle, ma.gaussians(), cams, vms, rcfg, wc, wd, None, ma.flat, ma.m, ma.v,
                                       acfg, step)
        abi.gs_render_fwd_batched(ctx.handle, mb.gaussians(), cams, vms, rcfg)
        abi.gs_render_bwd_batched(ctx.handle, mb.gaussians(), cams, vms, rcfg, wc, wd, None, mb.grads())
        abi.gs_adam_step(ctx.handle, mb.flat, mb.grad, mb.m, mb.v, mb.n, mb.sh_degree, acfg, step)
        torch.cuda.synchronize()
        for name, a, b in (("params", ma.flat, mb.flat), ("m", ma.m, mb.m), ("v", ma.v, mb.v)):
            a, b = a.cpu().numpy(), b.cpu().numpy()
            # float32 atomics order: a near-zero gradient can flip Adam's step sign
            bad = np.abs(a - b) > 1e-5 * np.abs(b) + 1e-7 * max(np.abs(b).max(), 1e-30)
            assert bad.sum() <= max(4, int(1e-4 * a.size)), (name, step, int(bad.sum()))


def test_batched_graph_replay_matches_eager(ctx):
    from paper_2408_12677_gb300.torch_api import BatchedTrainer, Context
    P, views = _mid_views(3)
    trgb = [_t(v.target_rgb) for v in views]
    tdep = [_t(v.target_depth) for v in views]
    vs = [(v.cam, v.pose.R, v.pose.t) for v in views]
    ma, mb = to_gpu_model(P), to_gpu_model(P)
    ea = BatchedTrainer(ma, vs, ctx=Context(0))
    eb = BatchedTrainer(mb, vs, ctx=Context(0))
    losses_a = []
    for _ in range(4):
        ea.step(trgb, tdep)
        losses_a.append(float(ea.loss.item()))
    eb.capture(trgb, tdep)  # runs one eager no-sync step first
    losses_b = [float(eb.loss.item())]
    for _ in range(3):
        eb.replay()
        torch.cuda.synchronize()
        losses_b.append(float(eb.loss.item()))
    eb.check_capacity()
    assert np.allclose(losses_a, losses_b, rtol=1e-4), (losses_a, losses_b)
    assert losses_a[-1] < losses_a[0]
    pa, pb = ma.flat.cpu().numpy(), mb.flat.cpu().numpy()
    assert np.abs(pa - pb).max() <= 1e-3 * np.abs(pa).max()


def test_batched_matches_sequential_iteration(ctx):
    """One batched iteration == the same iteration view by view (the
    comparison the batched form is measured against)."""
    from paper_2408_12677_gb300.torch_api import BatchedTrainer, Context
    P, views = _mid_views(3)
    trgb = [_t(v.target_rgb) for v in views]
    tdep = [_t(v.target_depth) for v in views]
    vs = [(v.cam, v.pose.R, v.pose.t) for v in views]
    ma, mb = to_gpu_model(P), to_gpu_model(P)
    ta = BatchedTrainer(ma, vs, ctx=Context(0))
    tb = BatchedTrainer(mb, vs, ctx=Context(0))
    for _ in range(2):
        la = float(ta.step(trgb, tdep).item())
        lb = float(tb.step_sequential(trgb, tdep).sum().item())
        assert abs(la - lb) <= 1e-5 * abs(lb)
    a, b = ma.flat.cpu().numpy(), mb.flat.cpu().numpy()
    bad = np.abs(a - b) > 1e-5 * np.abs(b) + 1e-6 * np.abs(b).max()
    assert bad.sum() <= max(4, int(1e-4 * a.size)), int(bad.sum())


def test_batched_argument_checks(ctx):
    from paper_2408_12677_gb300 import abi
    P, views = _mid_views(3)
    model = to_gpu_model(P)
    cams, vms = _structs(views)
    rcfg = abi.raster_cfg()
    with pytest.raises(abi.GsError) as e:
        abi.gs_render_fwd_batched(ctx.handle, model.gaussians(), [], [], rcfg)
    assert e.value.status == abi.GS_ERR_INVALID_ARG
    with pytest.raises(abi.GsError) as e:
        abi.gs_render_fwd_batched(ctx.handle, model.gaussians(), cams * 6, vms * 6, rcfg)  # 18 views
    assert e.value.status == abi.GS_ERR_INVALID_ARG
    abi.gs_render_fwd_batched(ctx.handle, model.gaussians(), cams, vms, rcfg)
    dc = [torch.zeros((3, v.cam.height, v.cam.width), device="cuda") for v in views]
    dd = [torch.zeros((v.cam.height, v.cam.width), device="cuda") for v in views]
    with pytest.raises(abi.GsError) as e:  # backward over other views than the forward's
        abi.gs_render_bwd_batched(ctx.handle, model.gaussians(), cams[:2], vms[:2], rcfg, dc[:2], dd[:2], None,
                                  model.grads())
    assert e.value.status == abi.GS_ERR_STATE
    torch.cuda.synchronize()


def test_autotune_picks_a_candidate_and_renders_the_same(ctx):
    from paper_2408_12677_gb300 import abi
    P, views = _mid_views(3)
    model = to_gpu_model(P)
    cams, vms = _structs(views)
    cfg = abi.raster_cfg()
    ms = abi.gs_autotune(ctx.handle, model.gaussians(), cams, vms, cfg, reps=2)
    assert len(ms) == 3 and all(m > 0 for m in ms)
    assert (cfg.tile_w, cfg.tile_h) in abi.AUTOTUNE_SHAPES
    assert ms[abi.AUTOTUNE_SHAPES.index((cfg.tile_w, cfg.tile_h))] == min(ms)
    # the tile shape changes the speed only: images of every candidate agree
    ref = _batched_render(ctx, model, views)
    for tw, th in abi.AUTOTUNE_SHAPES:
        for (c0, d0, a0), (c1, d1, a1) in zip(ref, _batched_render(ctx, model, views, tile_w=tw, tile_h=th)):
            assert np.abs(c0 - c1).max() <= 1e-5 and np.abs(d0 - d1).max() <= 1e-4 and np.abs(a0 - a1).max() <= 1e-5


def test_adam_step_device_counter(ctx):
    """gs_adam_step with step = 0 uses (and advances) the context's device step."""
    from paper_2408_12677_gb300 import abi
    P, _ = _mid_views(1)
    ma, mb = to_gpu_model(P), to_gpu_model(P)
    for mdl in (ma, mb):
        mdl.grad.copy_(torch.linspace(-1e-3, 1e-3, mdl.grad.numel(), device="cuda"))
    acfg = abi.adam_cfg(zero_grads=0)
    abi.gs_ctx_set_adam_step(ctx.handle, 4)
    abi.gs_adam_step(ctx.handle, ma.flat, ma.grad, ma.m, ma.v, ma.n, ma.sh_degree, acfg, 0)  # step 5
    abi.gs_adam_step(ctx.handle, ma.flat, ma.grad, ma.m, ma.v, ma.n, ma.sh_degree, acfg, 0)  # step 6
    abi.gs_adam_step(ctx.handle, mb.flat, mb.grad, mb.m, mb.v, mb.n, mb.sh_degree, acfg, 5)
    abi.gs_adam_step(ctx.handle, mb.flat, mb.grad, mb.m, mb.v, mb.n, mb.sh_degree, acfg, 6)
    torch.cuda.synchronize()
    a, b = ma.flat.cpu().numpy(), mb.flat.cpu().numpy()
    assert np.allclose(a, b, rtol=1e-6, atol=1e-7 * np.abs(b).max())
    abi.gs_ctx_set_adam_step(ctx.handle, 0)


def test_tile_visit_order_and_persistent_grid_change_nothing(ctx):
    """Longest-list-first tile order vs index order, persistent job-pulling
    grid vs one CTA per tile: identical forward images, gradients equal up to
    float32 atomics order."""
    from paper_2408_12677_gb300 import abi
    P, views = _mid_views(3)
    rng = np.random.default_rng(21)
    wc = [rng.standard_normal((3, v.cam.height, v.cam.width)).astype(np.float32) for v in views]
    wd = [rng.standard_normal((v.cam.height, v.cam.width)).astype(np.float32) for v in views]
    model = to_gpu_model(P)
    out = []
    for order, persistent in ((True, True), (False, False), (True, False), (False, True)):
        abi.gs_ctx_set_tile_order(ctx.handle, order)
        abi.gs_ctx_set_persistent(ctx.handle, persistent)
        imgs = _batched_render(ctx, model, views)
        out.append((imgs, _batched_backward(ctx, model, views, wc, wd, None)))
    abi.gs_ctx_set_tile_order(ctx.handle, True)
    abi.gs_ctx_set_persistent(ctx.handle, True)
    for other in out[1:]:
        for (c0, d0, a0), (c1, d1, a1) in zip(out[0][0], other[0]):
            assert np.array_equal(c0, c1) and np.array_equal(d0, d1) and np.array_equal(a0, a1)
        for k in NAMES:
            g0, g1 = out[0][1][k], other[1][k]
            compare(k, g0, g1, 1e-3, 1e-6 * np.abs(g1).max(), 1e-5, max(2, int(1e-3 * g1.size)))


def test_train_step_batched_matches_three_calls(ctx):
    from paper_2408_12677_gb300 import abi
    P, views = _mid_views(3)
    cams, vms = _structs(views)
    rcfg, acfg = abi.raster_cfg(), abi.adam_cfg()
    trgb = [_t(v.target_rgb) for v in views]
    tdep = [_t(v.target_depth) for v in views]
    A, B = to_gpu_model(P), to_gpu_model(P)
    shp = [((3, v.cam.height, v.cam.width), (v.cam.height, v.cam.width)) for v in views]
    col = [torch.empty(a, device="cuda") for a, _ in shp]
    dep = [torch.empty(b, device="cuda") for _, b in shp]
    dc = [torch.empty(a, device="cuda") for a, _ in shp]
    dd = [torch.empty(b, device="cuda") for _, b in shp]
    colB = [torch.empty(a, device="cuda") for a, _ in shp]
    depB = [torch.empty(b, device="cuda") for _, b in shp]
    la, lb = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
    for step in (1, 2):
        abi.gs_render_fwd_batched(ctx.handle, A.gaussians(), cams, vms, rcfg, col, dep, None)
        abi.gs_loss_l1_batched(ctx.handle, cams, col, dep, trgb, tdep, 0.8, 0.2, la, dc, dd)
        abi.gs_render_bwd_adam_batched(ctx.handle, A.gaussians(), cams, vms, rcfg, dc, dd, None, A.flat, A.m, A.v,
                                       acfg, step)
        abi.gs_train_step_batched(ctx.handle, B.gaussians(), cams, vms, rcfg, trgb, tdep, 0.8, 0.2, lb, B.flat, B.m,
                                  B.v, acfg, step, colB, depB, None)
        torch.cuda.synchronize()
        if step == 1:  # same map: the rendered images are bit-identical
            for x, y in zip(col + dep, colB + depB):
                assert torch.equal(x, y)
        assert abs(float(la.item()) - float(lb.item())) <= 1e-6 * abs(float(la.item()))
        for name, x, y in (("p", A.flat, B.flat), ("m", A.m, B.m), ("v", A.v, B.v)):
            xa, ya = x.cpu().numpy(), y.cpu().numpy()
            bad = np.abs(xa - ya) > 1e-5 * np.abs(xa) + 1e-6 * np.abs(xa).max() + 1e-12
            assert bad.sum() <= max(4, int(1e-4 * xa.size)), (name, step, int(bad.sum()))


def test_visit_order_with_many_tiles(ctx):
    """Two 1200x680 views (6450 tiles: the multi-block binning scan builds the
    visit order): the same images with and without the order and with a CTA
    per tile, so the order is a permutation of all tiles."""
    from paper_2408_12677_gb300 import abi
    rng = np.random.default_rng(41)
    views = []
    for k, eye in enumerate(([0.0, 0.0, 0.0], [0.2, -0.3, 0.1])):
        cam = Camera(600.0, 600.0, 600.0, 340.0, 1200, 680)
        views.append(workloads.View(cam, look_at(eye, [2.5, 0.0, 0.0]), None, None))
    P = workloads.random_gaussians(rng, 40000, views[0].cam, views[0].pose, 0, z_range=(1.5, 3.5),
                                   log_scale_range=(-4.0, -2.0))
    model = to_gpu_model(P)
    out = []
    for order, persistent in ((True, True), (False, True), (True, False)):
        abi.gs_ctx_set_tile_order(ctx.handle, order)
        abi.gs_ctx_set_persistent(ctx.handle, persistent)
        out.append(_batched_render(ctx, model, views))
    abi.gs_ctx_set_tile_order(ctx.handle, True)
    abi.gs_ctx_set_persistent(ctx.handle, True)
    assert ctx.stats()["n_tiles"] == 2 * 75 * 43
    for other in out[1:]:
        for (c0, d0, a0), (c1, d1, a1) in zip(out[0], other):
            assert np.array_equal(c0, c1) and np.array_equal(d0, d1) and np.array_equal(a0, a1)
    assert float(np.mean(out[0][0][2] > 0.1)) > 0.3  # the views see the cloud
