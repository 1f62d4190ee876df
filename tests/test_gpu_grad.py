"""Backward pass on the GPU vs the oracle's autograd gradients (and, for the
autograd Function, vs central differences of the GPU forward).

Gradient tolerance: per parameter array ||g - o|| / ||o|| <= 1e-3 and
element-wise |g - o| <= 1e-3 |o| + 1e-5 max|o| (the largest error measured
over every scene here is 2.3% of that bound).  Elements beyond it are flips:
the Gaussian must have a
float32 decision within 1e-4 (relative) of its threshold at some pixel it
reaches (``R.decision_margins``, reported with the threshold), and there may
be at most max(1, 1e-5 x elements) of them per array (the census of every
scene here found none).  Arrays whose exact gradient is 0 are checked against
the floor only."""
import numpy as np
import pytest
import torch

from oracle import render as R
from synth import workloads
from synth.scene import Camera, Pose, look_at
from tests._util import compare, ensure_built, gpu_backward, gpu_render, to_gpu_model

pytestmark = pytest.mark.gpu

NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


@pytest.fixture(scope="module")
def ctx():
    ensure_built()
    from paper_2408_12677_gb300.torch_api import Context
    c = Context(0)
    yield c
    c.close()


def _all_pixels(cam):
    jj, ii = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    return np.stack([ii.ravel(), jj.ravel()], 1)


def _check_grads(ctx, P, deg, cam, pose, seed, with_alpha=True, **cfg):
    rng = np.random.default_rng(seed)
    H, W = cam.height, cam.width
    wc = rng.standard_normal((3, H, W)).astype(np.float32)
    wd = rng.standard_normal((H, W)).astype(np.float32)
    wa = rng.standard_normal((H, W)).astype(np.float32) if with_alpha else None
    model = to_gpu_model(P)
    gpu_render(ctx, model, cam, pose, **cfg)
    g = gpu_backward(ctx, model, cam, pose, wc, wd, wa, **cfg)
    R64, t64 = pose.R.astype(np.float64), pose.t.astype(np.float64)
    og, _ = R.weighted_pixel_gradients(P, deg, cam, R64, t64, _all_pixels(cam), wc.reshape(3, -1).astype(np.float64),
                                       wd.reshape(-1).astype(np.float64),
                                       None if wa is None else wa.reshape(-1).astype(np.float64), prefilter=True)
    m = R.decision_margins(P, deg, cam, R64, t64)
    check_grad_arrays(g, og, m)


GRAD_FLIP_GAUSSIANS = 0  # whole Gaussians' gradients allowed to flip on top of max(1, 1e-5 x elements)


def check_grad_arrays(g, og, margins=None, names=NAMES + ("pose",), flip_gaussians=GRAD_FLIP_GAUSSIANS,
                      report=None):
    G = max(float(np.abs(og[k].detach().numpy()).max(initial=0.0)) for k in NAMES)
    for k in names:
        ref = og[k].detach().numpy()
        scale = np.abs(ref).max(initial=0.0)
        floor = 1e-5 * scale + 1e-12
        if scale <= 1e-6 * G:  # exact gradient is (numerically) zero
            assert np.abs(g[k]).max(initial=0.0) <= 1e-5 * G, (k, np.abs(g[k]).max())
            continue
        mk = {}
        n_g = max(ref.shape[0], 1)
        per = ref.size // n_g
        if margins is not None and k != "pose":
            # flips are decisions of single Gaussians (within flip_eps of a
            # threshold): the budget counts flipped Gaussians, each of which
            # moves up to `per` elements
            mk = dict(margins=np.repeat(margins["gauss"], per), kinds=np.repeat(margins["gauss_kind"], per),
                      groups=np.repeat(np.arange(n_g), per))
            budget = max(1, int(1e-5 * n_g)) + flip_gaussians
        else:
            budget = 0 if k == "pose" else max(1, int(1e-5 * ref.size)) + flip_gaussians * per
        compare(k, g[k], ref, 1e-3, floor, 1e-3, budget, report, **mk)


def test_tiny_random_gradients(ctx):
    w = workloads.tiny_random(seed=1000)
    _check_grads(ctx, w.params, 0, w.views[0].cam, w.views[0].pose, 1)


@pytest.mark.parametrize("tile", [(8, 32), (32, 8)])
def test_gradients_sh3_posed(ctx, tile):
    cam = Camera(80.0, 75.0, 40.0, 30.0, 84, 60)
    pose = look_at([0.1, 0.2, -0.1], [0.7, 3.0, 0.2])
    P = workloads.random_gaussians(np.random.default_rng(5), 700, cam, pose, 3, log_scale_range=(-3.5, -1.5),
                                   sh_rest_std=0.15)
    _check_grads(ctx, P, 3, cam, pose, 2, tile_w=tile[0], tile_h=tile[1])


def test_gradients_without_alpha_upstream(ctx):
    w = workloads.tiny_random(seed=1001, n=300, sh_degree=1, sh_rest_std=0.2)
    _check_grads(ctx, w.params, 1, w.views[0].cam, w.views[0].pose, 3, with_alpha=False)


def test_autograd_function_matches_abi_and_fd(ctx):
    from paper_2408_12677_gb300.torch_api import render
    cam = Camera(40.0, 40.0, 20.0, 16.0, 40, 32)
    pose = look_at([0.0, 0.0, 0.0], [0.2, 3.0, 0.1])
    P = workloads.random_gaussians(np.random.default_rng(11), 60, cam, pose, 3, z_range=(1.0, 2.5),
                                   log_scale_range=(-2.6, -1.8), sh_rest_std=0.1)
    T = {k: torch.tensor(np.asarray(P[k], np.float32), device="cuda", requires_grad=True) for k in NAMES}
    xi = torch.zeros(6, requires_grad=True)
    rng = np.random.default_rng(4)
    wc = torch.tensor(rng.standard_normal((3, 32, 40)), dtype=torch.float32, device="cuda")
    wd = torch.tensor(rng.standard_normal((32, 40)), dtype=torch.float32, device="cuda")
    col, dep, alp = render(ctx, T, 3, cam, pose.R, pose.t, pose_xi=xi)
    obj = (col * wc).sum() + (dep * wd).sum()
    obj.backward()
    og, _ = R.weighted_pixel_gradients(P, 3, cam, pose.R.astype(np.float64), pose.t.astype(np.float64),
                                       _all_pixels(cam), wc.cpu().numpy().reshape(3, -1).astype(np.float64),
                                       wd.cpu().numpy().reshape(-1).astype(np.float64), None)
    got = {k: T[k].grad.cpu().numpy() for k in NAMES}
    got["pose"] = xi.grad.numpy()
    check_grad_arrays(got, og, R.decision_margins(P, 3, cam, pose.R.astype(np.float64), pose.t.astype(np.float64)))
    # central differences of the float32 GPU forward on a few large gradient entries
    for k in ("means", "log_scales", "opacity_logits", "sh"):
        g = T[k].grad.reshape(-1)
        i = int(torch.argmax(g.abs()))
        h = 2e-3
        vals = []
        for s in (1.0, -1.0):
            with torch.no_grad():
                T2 = {kk: vv.detach().clone() for kk, vv in T.items()}
                T2[k].reshape(-1)[i] += s * h
                c2, d2, _ = render(ctx, T2, 3, cam, pose.R, pose.t)
                vals.append(float((c2 * wc).sum() + (d2 * wd).sum()))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - float(g[i])) <= 3e-2 * abs(float(g[i])) + 1e-3, (k, fd, float(g[i]))


def test_two_renders_of_one_map_then_backward(ctx):
    """The forward state (Sec. III-B.3: each backward pass belongs to its own
    forward pass): two differentiable renders of one map at two poses summed
    into one objective give the oracle's two-view gradient (the second
    render's state replaced the first's; the autograd Function sees the token
    change and recomputes), and through the raw ABI a backward pass of the
    first pose after the second forward pass fails with GS_ERR_STATE."""
    from paper_2408_12677_gb300 import abi
    from paper_2408_12677_gb300.torch_api import render
    from tests._util import margins_over_views
    cam = Camera(48.0, 48.0, 24.0, 18.0, 48, 36)
    poses = [look_at([0.0, 0.0, 0.0], [0.2, 3.0, 0.1]), look_at([0.15, -0.1, 0.05], [0.1, 3.0, 0.2])]
    P = workloads.random_gaussians(np.random.default_rng(12), 120, cam, poses[0], 1, z_range=(1.2, 2.8),
                                   log_scale_range=(-2.6, -1.8), sh_rest_std=0.1)
    T = {k: torch.tensor(np.asarray(P[k], np.float32), device="cuda", requires_grad=True) for k in NAMES}
    rng = np.random.default_rng(8)
    wc = [torch.tensor(rng.standard_normal((3, 36, 48)), dtype=torch.float32, device="cuda") for _ in poses]
    wd = [torch.tensor(rng.standard_normal((36, 48)), dtype=torch.float32, device="cuda") for _ in poses]
    outs = [render(ctx, T, 1, cam, p.R, p.t) for p in poses]
    obj = sum((c * a).sum() + (d * b).sum() for (c, d, _), a, b in zip(outs, wc, wd))
    obj.backward()
    p64 = [(p.R.astype(np.float64), p.t.astype(np.float64)) for p in poses]
    og = R.multiview_weighted_gradients(P, 1, [cam, cam], p64, [x.cpu().numpy().astype(np.float64) for x in wc],
                                        [x.cpu().numpy().astype(np.float64) for x in wd], with_pose=False)
    got = {k: T[k].grad.cpu().numpy() for k in NAMES}
    check_grad_arrays(got, og, margins_over_views(P, 1, [cam, cam], p64), names=NAMES)
    # raw ABI: the state is the last forward pass's; another pose is refused
    model = to_gpu_model(P)
    gpu_render(ctx, model, cam, poses[0])
    t0 = abi.gs_state_token(ctx.handle)
    gpu_render(ctx, model, cam, poses[1])
    t1 = abi.gs_state_token(ctx.handle)
    assert t0 != 0 and t1 != 0 and t0 != t1
    z = np.zeros((36, 48), np.float32)
    with pytest.raises(abi.GsError) as e:
        gpu_backward(ctx, model, cam, poses[0], np.zeros((3, 36, 48), np.float32), z, None)
    assert e.value.status == abi.GS_ERR_STATE
    # another raster configuration or other parameter arrays are refused too
    with pytest.raises(abi.GsError) as e:
        gpu_backward(ctx, model, cam, poses[1], np.zeros((3, 36, 48), np.float32), z, None, tile_w=8, tile_h=32)
    assert e.value.status == abi.GS_ERR_STATE
    with pytest.raises(abi.GsError) as e:
        gpu_backward(ctx, to_gpu_model(P), cam, poses[1], np.zeros((3, 36, 48), np.float32), z, None)
    assert e.value.status == abi.GS_ERR_STATE
    gpu_backward(ctx, model, cam, poses[1], np.zeros((3, 36, 48), np.float32), z, None)  # its own state: fine
