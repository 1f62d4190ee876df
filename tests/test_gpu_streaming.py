"""The per-frame streaming loop on the GPU: the map grows only where it does
not cover a frame yet, doubles its capacity without disturbing live slots,
keeps inert slots inert, and its batched gradients at checkpoints match the
FP64 oracle (and central differences of the oracle loss, h = 1e-4)."""
import numpy as np
import pytest
import torch

from oracle import render as R
from synth import workloads
from synth.quadtree import seed_gaussians
from tests._util import ensure_built, margins_over_views, residual_margins
from tests.test_gpu_grad import check_grad_arrays

pytestmark = pytest.mark.gpu

NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")
DEG = 1


def _seed(rgb, depth, cam, pose, mask):
    return seed_gaussians(rgb, depth, cam, pose, DEG, var_thr=0.03, min_size=4, mask=mask)


@pytest.fixture(scope="module")
def run():
    ensure_built()
    from paper_2408_12677_gb300.streaming import StreamingOptimizer
    st = workloads.streaming(n_frames=8, width=96, height=64, f=48.0)
    frames = [st.frame(k) for k in range(6)]
    opt = StreamingOptimizer(st.cam, DEG, _seed, iters=3, n_past=2, capacity=256, rng_seed=1)
    stats = [opt.process_frame(rgb, dep, st.poses[k]) for k, (rgb, dep) in enumerate(frames)]
    return st, frames, opt, stats


def test_map_grows_where_uncovered_and_capacity_doubles(run):
    st, frames, opt, stats = run
    ns = [s.n_gaussians for s in stats]
    assert ns[0] > 200 and all(b >= a for a, b in zip(ns, ns[1:]))
    assert stats[-1].capacity > 256 and stats[-1].capacity >= ns[-1]
    assert stats[0].keyframe and all(np.isfinite(s.loss) for s in stats)
    # the last frame again: its pixels are covered now, so it seeds far fewer Gaussians
    rgb, dep = frames[-1]
    again = opt.process_frame(rgb, dep, st.poses[len(frames) - 1])
    assert again.new_gaussians < 0.2 * stats[0].new_gaussians, (again.new_gaussians, stats[0].new_gaussians)
    m = opt.map.model
    n = opt.map.n
    assert torch.isfinite(m.flat).all()
    assert bool((m.p["opacity_logits"][n:] == -30.0).all()) and bool((m.p["log_scales"][n:] == -30.0).all())
    from paper_2408_12677_gb300.torch_api import flat_sizes
    off = 0
    for size in flat_sizes(m.n, DEG):  # inert slots never get Adam state
        per = size // m.n
        assert float(m.m[off + n * per:off + size].abs().max()) == 0.0
        assert float(m.v[off + n * per:off + size].abs().max()) == 0.0
        off += size


def test_checkpoint_gradients_match_oracle(run):
    """The batched gradient of the current frame + two keyframes against the
    FP64 oracle's multi-view gradient, on the live slots of the grown map."""
    from paper_2408_12677_gb300 import abi
    st, frames, opt, stats = run
    views = [opt.keyframes[-1], opt.keyframes[0]] + ([opt.keyframes[1]] if len(opt.keyframes) > 2 else [])
    h = opt.ctx.handle
    m = opt.map.model
    V = len(views)
    cams = [opt.cam_s] * V
    vms = [k.view for k in views]
    abi.gs_render_fwd_batched(h, m.gaussians(), cams, vms, opt.rcfg, opt.color[:V], opt.depth[:V], opt.alpha[:V])
    abi.gs_loss_l1_batched(h, cams, opt.color[:V], opt.depth[:V], [k.rgb for k in views], [k.depth for k in views],
                           0.8, 0.2, opt.loss, opt.dLdc[:V], opt.dLdd[:V])
    m.grad.zero_()
    gp = torch.zeros((V, 6), device="cuda")
    abi.gs_render_bwd_batched(h, m.gaussians(), cams, vms, opt.rcfg, opt.dLdc[:V], opt.dLdd[:V], None, m.grads(), gp)
    torch.cuda.synchronize()
    n = opt.map.n
    g = {k: v[:n].detach().cpu().numpy().copy() for k, v in m.g.items()}
    for k, v in m.g.items():
        assert float(v[n:].abs().max()) == 0.0, k  # inert slots: exactly no gradient
    g["pose"] = gp.cpu().numpy()
    P = opt.map.live_params()
    poses = [(np.array(k.view.R, np.float64).reshape(3, 3), np.array(k.view.t, np.float64)) for k in views]
    targets = [(k.rgb.cpu().numpy(), k.depth.cpu().numpy()) for k in views]
    L, og_loss, _ = R.multiview_gradients(P, DEG, [st.cam] * V, poses, targets)
    assert abs(float(opt.loss.item()) - float(L)) <= 1e-4 * float(L)
    # the backward pass against the oracle's, both driven by the image
    # gradients the GPU loss wrote (so an L1 sign that flips at a residual
    # near 0 does not enter the comparison; the loss is compared above)
    wc = [x.cpu().numpy().astype(np.float64) for x in opt.dLdc[:V]]
    wd = [x.cpu().numpy().astype(np.float64) for x in opt.dLdd[:V]]
    og = R.multiview_weighted_gradients(P, DEG, [st.cam] * V, poses, wc, wd)
    check_grad_arrays(g, og, margins_over_views(P, DEG, [st.cam] * V, poses))
    og = og_loss  # central differences below are of the loss itself

    # central differences of the FP64 loss (h = 1e-4) at the largest gradient entries
    Pd = {k: (np.asarray(v, np.float64) if isinstance(v, np.ndarray) else v) for k, v in P.items()}
    checked = 0
    for name in ("means", "log_scales", "opacity_logits", "sh"):
        G = og[name].numpy().ravel()
        for i in np.argsort(-np.abs(G))[:3]:
            def f(hh):
                Q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in Pd.items()}
                Q[name].reshape(-1)[i] += hh
                T = R.to_tensors(Q)
                with torch.no_grad():
                    return sum(float(R.render_loss(T, DEG, st.cam, Rm, tv, trgb, tdep)[0])
                               for (Rm, tv), (trgb, tdep) in zip(poses, targets))
            d1 = (f(1e-4) - f(-1e-4)) / 2e-4
            d2 = (f(5e-5) - f(-5e-5)) / 1e-4
            if abs(d1 - d2) > 1e-3 * max(abs(d1), abs(d2), 1e-9):
                continue  # a kink (L1 sign, support edge) within h
            gpu = g[name].ravel()[i]
            assert abs(gpu - d1) <= 2e-3 * abs(d1) + 1e-6 * np.abs(G).max(), (name, i, gpu, d1)
            checked += 1
    assert checked >= 6


def test_global_optimisation_step_matches_oracle(run):
    """One step of the offline optimisation over the keyframe list (Sec.
    III-B.3): the loss summed over every keyframe (one batched step) and the
    Adam update it makes, against the FP64 oracle's multi-view loss, its
    gradient and the float64 Adam step from the same parameters and moments
    (with the float32 hyper-parameters the ABI receives)."""
    from oracle import adam as oadam
    from paper_2408_12677_gb300.streaming import global_optimize
    from paper_2408_12677_gb300.torch_api import _views
    from tests._util import compare
    st, frames, opt, stats = run
    kfs = opt.keyframes
    assert 2 <= len(kfs) <= 16
    m = opt.map.model
    n, cap = opt.map.n, m.n
    names = R.PARAM_NAMES

    def live(flat):
        return {k: v[:n].detach().cpu().numpy().astype(np.float64).copy() for k, v in _views(flat, cap, DEG).items()}

    P0, M0, V0 = live(m.flat), live(m.m), live(m.v)
    inert0 = m.flat.clone()
    g = global_optimize(opt, epochs=1, views_per_step=len(kfs), rng_seed=7)
    assert g.steps == 1 and g.view_iterations == len(kfs)
    P1 = live(m.flat)
    # inert slots are untouched
    for k, v in _views(m.flat, cap, DEG).items():
        assert torch.equal(v[n:], _views(inert0, cap, DEG)[k][n:]), k
    poses = [(np.array(k.view.R, np.float64).reshape(3, 3), np.array(k.view.t, np.float64)) for k in kfs]
    targets = [(k.rgb.cpu().numpy(), k.depth.cpu().numpy()) for k in kfs]
    P = dict(P0, sh_degree=DEG)
    L, og, outs = R.multiview_gradients(P, DEG, [st.cam] * len(kfs), poses, targets, with_pose=False)
    assert abs(g.loss_first - float(L)) <= 1e-4 * float(L), (g.loss_first, float(L))
    # where a loss residual is within float32 rounding of 0 its sign (the
    # image gradient) may flip: such pixels flag the Gaussians they reach
    extras = [residual_margins(o["color"].detach().numpy(), o["depth"].detach().numpy(), trgb, tdep)
              for o, (trgb, tdep) in zip(outs, targets)]
    mg = margins_over_views(P, DEG, [st.cam] * len(kfs), poses, extras)
    f32 = lambda x: float(np.float32(x))
    a = opt.acfg
    cfg = oadam.AdamCfg(f32(a.lr_means), f32(a.lr_log_scales), f32(a.lr_quats), f32(a.lr_opacity), f32(a.lr_sh_dc),
                        f32(a.lr_sh_rest), f32(a.beta1), f32(a.beta2), f32(a.eps))
    flat = lambda d: np.concatenate([np.asarray(d[k], np.float64).ravel() for k in names])
    lr = oadam.lr_per_element(n, DEG, cfg)
    gflat = flat({k: og[k].numpy() for k in names})
    p_new, _, v_new = oadam.adam_step(flat(P0), gflat, flat(M0), flat(V0), opt.step, lr, cfg)
    d_gpu, d_ref = flat(P1) - flat(P0), p_new - flat(P0)
    # the tolerance is the gradient tolerance (1e-3 |g| + 1e-5 max|g| per
    # array) carried through Adam: a gradient error dg moves the first moment
    # by (1 - b1) dg, hence the step by lr (1 - b1) / (1 - b1^t) dg /
    # (sqrt(v^) + eps) -- large where the moment cancels -- plus 1e-3 of the
    # step for the second moment's share
    gmax = np.concatenate([np.full(og[k].numpy().size, np.abs(og[k].numpy()).max()) for k in names])
    dg = 1e-3 * np.abs(gflat) + 1e-5 * gmax
    vhat = v_new / (1.0 - cfg.beta2 ** opt.step)
    atol = lr * (1.0 - cfg.beta1) / (1.0 - cfg.beta1 ** opt.step) * dg / (np.sqrt(vhat) + cfg.eps)
    # the GPU stores the updated parameter in float32: its step is a
    # difference of two float32 values, rounded to a unit in the last place
    atol = atol + np.spacing(np.abs(p_new).astype(np.float32)).astype(np.float64)
    per = {k: og[k].numpy().size // n for k in names}
    mrg = np.concatenate([np.repeat(mg["gauss"], per[k]) for k in names])
    knd = np.concatenate([np.repeat(mg["gauss_kind"], per[k]) for k in names])
    # every element beyond the tolerance must belong to a flagged Gaussian
    from tests._util import FLIP_EPS
    budget = max(1, int(1e-5 * d_ref.size)) + int((mrg <= FLIP_EPS).sum())
    compare("adam update", d_gpu, d_ref, 1e-3, atol, 1e-3, budget, margins=mrg, kinds=knd)


def test_global_optimisation_over_keyframes(run):
    """The offline pass over the keyframe list: every keyframe visited once per
    epoch in batches of up to 16 views, finite map, the summed loss of a
    fixed batch decreases."""
    from paper_2408_12677_gb300 import abi
    from paper_2408_12677_gb300.streaming import global_optimize
    st, frames, opt, stats = run
    kfs = opt.keyframes
    probe = kfs[: min(4, len(kfs))]

    def probe_loss():
        V = len(probe)
        abi.gs_render_fwd_batched(opt.ctx.handle, opt.map.model.gaussians(), [opt.cam_s] * V, [k.view for k in probe],
                                  opt.rcfg, opt.color[:V], opt.depth[:V], None)
        abi.gs_loss_l1_batched(opt.ctx.handle, [opt.cam_s] * V, opt.color[:V], opt.depth[:V], [k.rgb for k in probe],
                               [k.depth for k in probe], 0.8, 0.2, opt.loss, opt.dLdc[:V], opt.dLdd[:V])
        return float(opt.loss.item())

    before = probe_loss()
    g = global_optimize(opt, epochs=3, views_per_step=3, rng_seed=2)
    after = probe_loss()
    assert g.keyframes == len(kfs) and g.view_iterations == 3 * len(kfs)
    assert g.steps == 3 * -(-len(kfs) // 3)
    assert torch.isfinite(opt.map.model.flat).all()
    assert after < before, (before, after)
