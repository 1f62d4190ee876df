"""Pins for the oracle's gradients: torch.autograd through the FP64 forward vs
central finite differences of that forward (h and h/2; points where the two
differences disagree straddle a kink of the piecewise-smooth image -- the
3-sigma edge, the 1/255 skip, the transmittance stop, the 0.99 clamp or an
L1 sign change -- and are skipped and counted)."""
import numpy as np
import pytest
import torch

from oracle import render as R
from synth import workloads
from synth.scene import Camera, look_at

DT = torch.float64
CAM = Camera(30.0, 28.0, 16.0, 12.0, 32, 24)


def _scene(seed, n=28, deg=3):
    rng = np.random.default_rng(seed)
    pose = look_at([0.2, -0.1, 0.05], [0.5, 3.0, 0.3])
    P = workloads.random_gaussians(rng, n, CAM, pose, deg, z_range=(0.8, 2.5),
                                   log_scale_range=(-2.8, -1.6), sh_rest_std=0.15)
    P = {k: (np.asarray(v, np.float64) if isinstance(v, np.ndarray) else v) for k, v in P.items()}
    P["opacity_logits"] = rng.uniform(-1.0, 2.5, n)
    return P, pose


def _objective(P, deg, pose, xi, wc, wd, wa):
    T = R.to_tensors(P)
    Rm, t = R.perturb_pose(torch.as_tensor(pose.R, dtype=DT), torch.as_tensor(pose.t, dtype=DT), xi)
    out = R.render(T, deg, CAM, Rm, t)
    return float((out["color"] * wc).sum() + (out["depth"] * wd).sum() + (out["alpha"] * wa).sum())


def _fd_check(f, analytic, coords, h):
    ok, kinks = 0, 0
    for idx, g in zip(coords, analytic):
        d1 = (f(idx, h) - f(idx, -h)) / (2 * h)
        d2 = (f(idx, h / 2) - f(idx, -h / 2)) / h
        if abs(d1 - d2) > 1e-3 * max(abs(d1), abs(d2), 1e-6):
            kinks += 1
            continue
        assert abs(g - d1) <= 1e-5 * abs(d1) + 1e-7, (idx, g, d1)
        ok += 1
    return ok, kinks


@pytest.mark.parametrize("seed", [21, 22])
def test_linear_objective_gradients_match_fd(seed):
    P, pose = _scene(seed)
    deg = 3
    rng = np.random.default_rng(seed + 100)
    wc = torch.as_tensor(rng.standard_normal((3, CAM.height, CAM.width)))
    wd = torch.as_tensor(rng.standard_normal((CAM.height, CAM.width)))
    wa = torch.as_tensor(rng.standard_normal((CAM.height, CAM.width)))
    pix = np.stack(np.meshgrid(np.arange(CAM.width), np.arange(CAM.height), indexing="xy"), -1).reshape(-1, 2)
    grads, _ = R.weighted_pixel_gradients(P, deg, CAM, pose.R, pose.t, pix, wc.reshape(3, -1), wd.reshape(-1),
                                          wa.reshape(-1), prefilter=False)
    zero_xi = torch.zeros(6, dtype=DT)
    total_ok = 0
    for name in R.PARAM_NAMES:
        G = grads[name].numpy()
        flat = np.flatnonzero(np.abs(G.ravel()) > 1e-8)
        assert flat.size > 0, name
        pick = rng.choice(flat, min(8, flat.size), replace=False)

        def f(i, h, name=name):
            Q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in P.items()}
            Q[name].reshape(-1)[i] += h
            return _objective(Q, deg, pose, zero_xi, wc, wd, wa)

        ok, kinks = _fd_check(f, G.ravel()[pick], pick, 1e-6)
        assert ok >= len(pick) - 2, (name, ok, kinks)
        total_ok += ok
    gp = grads["pose"].numpy()

    def fpose(i, h):
        xi = torch.zeros(6, dtype=DT)
        xi[i] = h
        return _objective(P, deg, pose, xi, wc, wd, wa)

    ok, kinks = _fd_check(fpose, gp, range(6), 1e-6)
    assert ok >= 5, (ok, kinks)


def test_l1_loss_gradients_match_fd():
    P, pose = _scene(31)
    deg = 3
    rng = np.random.default_rng(5)
    trgb = rng.uniform(0, 1, (3, CAM.height, CAM.width))
    tdep = rng.uniform(0.5, 3.0, (CAM.height, CAM.width))
    tdep[:3] = 0.0
    L, grads, _ = R.gradients(P, deg, CAM, pose.R, pose.t, trgb, tdep)

    def loss(Q, xi):
        T = R.to_tensors(Q)
        Rm, t = R.perturb_pose(torch.as_tensor(pose.R, dtype=DT), torch.as_tensor(pose.t, dtype=DT), xi)
        return float(R.render_loss(T, deg, CAM, Rm, t, trgb, tdep)[0])

    assert abs(loss(P, torch.zeros(6, dtype=DT)) - float(L)) < 1e-14
    for name in ("means", "log_scales", "opacity_logits", "sh"):
        G = grads[name].numpy()
        flat = np.flatnonzero(np.abs(G.ravel()) > 1e-9)
        pick = rng.choice(flat, min(6, flat.size), replace=False)

        def f(i, h, name=name):
            Q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in P.items()}
            Q[name].reshape(-1)[i] += h
            return loss(Q, torch.zeros(6, dtype=DT))

        ok, kinks = _fd_check(f, G.ravel()[pick], pick, 1e-6)
        assert ok >= len(pick) - 2, (name, ok, kinks)

    def fpose(i, h):
        xi = torch.zeros(6, dtype=DT)
        xi[i] = h
        return loss(P, xi)

    ok, kinks = _fd_check(fpose, grads["pose"].numpy(), range(6), 1e-6)
    assert ok >= 5, (ok, kinks)


def test_clamped_alpha_has_zero_opacity_gradient():
    """alpha = min(0.99, o G): where the clamp is active the opacity gets no
    gradient from that pixel."""
    sc = {"means": np.array([[0.0, 0.0, 1.0]]), "log_scales": np.full((1, 3), np.log(3.0)),
          "quats": np.array([[1.0, 0, 0, 0]]), "opacity_logits": np.array([12.0]), "sh": np.zeros((1, 1, 3))}
    pix = np.array([[16, 12]])
    g, out = R.weighted_pixel_gradients(sc, 0, CAM, np.eye(3), np.zeros(3), pix, np.ones((3, 1)), np.ones(1),
                                        np.ones(1), with_pose=False)
    assert abs(float(out["alpha"].detach()[0]) - 0.99) < 1e-15
    assert float(g["opacity_logits"][0]) == 0.0
