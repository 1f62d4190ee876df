"""Pins for the oracle's multi-view objective (batched form: the loss of one
batched iteration is the sum of the per-view losses, each normalised by its
own pixel count; one Adam step then uses the summed gradient).

The pins tie it to things other than its own code path: the single-view
definition (one view, duplicated views, a permutation of the views),
central finite differences of the summed loss, and the chain rule through
the per-view loss image gradients (``multiview_weighted_gradients``)."""
import numpy as np
import pytest
import torch

from oracle import render as R
from synth import workloads

DT = torch.float64


@pytest.fixture(scope="module")
def scene():
    w = workloads.tiny_multi_view(seed=1005, n=40, sh_degree=1, sh_rest_std=0.1,
                                  cams=((24, 18, 24.0), (16, 12, 18.0), (20, 14, 22.0)))
    P = {k: (np.asarray(v, np.float64) if isinstance(v, np.ndarray) else v) for k, v in w.params.items()}
    return w, P


def _args(w, idx):
    cams = [w.views[i].cam for i in idx]
    poses = [(w.views[i].pose.R.astype(np.float64), w.views[i].pose.t.astype(np.float64)) for i in idx]
    targets = [(w.views[i].target_rgb, w.views[i].target_depth) for i in idx]
    return cams, poses, targets


def _close(a, b, rtol=1e-12):
    a, b = np.asarray(a), np.asarray(b)
    assert np.allclose(a, b, rtol=rtol, atol=rtol * max(np.abs(b).max(initial=0.0), 1e-300)), \
        float(np.abs(a - b).max(initial=0.0))


def test_one_view_is_the_single_view_definition(scene):
    w, P = scene
    cams, poses, targets = _args(w, [1])
    L, g, _ = R.multiview_gradients(P, 1, cams, poses, targets)
    v = w.views[1]
    L1, g1, _ = R.gradients(P, 1, v.cam, poses[0][0], poses[0][1], v.target_rgb, v.target_depth)
    _close(L, L1)
    for k in R.PARAM_NAMES:
        _close(g[k].numpy(), g1[k].numpy())
    _close(g["pose"][0].numpy(), g1["pose"].numpy())


def test_sum_over_views_and_permutation(scene):
    w, P = scene
    L012, g012, _ = R.multiview_gradients(P, 1, *_args(w, [0, 1, 2]))
    L201, g201, _ = R.multiview_gradients(P, 1, *_args(w, [2, 0, 1]))
    singles = [R.multiview_gradients(P, 1, *_args(w, [i])) for i in range(3)]
    _close(L012, sum(s[0] for s in singles), 1e-13)
    _close(L201, L012, 1e-13)
    for k in R.PARAM_NAMES:
        total = sum(s[1][k].numpy() for s in singles)
        _close(g012[k].numpy(), total, 1e-11)
        _close(g201[k].numpy(), g012[k].numpy(), 1e-11)
    # pose gradients belong to their own view
    for i in range(3):
        _close(g012["pose"][i].numpy(), singles[i][1]["pose"][0].numpy(), 1e-12)
    _close(g201["pose"].numpy(), g012["pose"].numpy()[[2, 0, 1]], 1e-12)


def test_duplicated_view_doubles(scene):
    w, P = scene
    L, g, _ = R.multiview_gradients(P, 1, *_args(w, [0, 0]))
    L1, g1, _ = R.multiview_gradients(P, 1, *_args(w, [0]))
    _close(L, 2 * L1, 1e-13)
    for k in R.PARAM_NAMES:
        _close(g[k].numpy(), 2 * g1[k].numpy(), 1e-12)


def test_summed_loss_matches_finite_differences(scene):
    w, P = scene
    cams, poses, targets = _args(w, [0, 1, 2])
    L, g, _ = R.multiview_gradients(P, 1, cams, poses, targets, with_pose=False)
    rng = np.random.default_rng(7)

    def loss_at(Q):
        return float(R.multiview_gradients(Q, 1, cams, poses, targets, with_pose=False)[0])

    checked = 0
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        G = g[k].numpy().ravel()
        cand = np.flatnonzero(np.abs(G) > 1e-6 * np.abs(G).max())
        for i in rng.choice(cand, min(5, cand.size), replace=False):
            def f(h):
                Q = {kk: (v.copy() if isinstance(v, np.ndarray) else v) for kk, v in P.items()}
                Q[k].reshape(-1)[i] += h
                return loss_at(Q)
            h = 1e-4
            d1 = (f(h) - f(-h)) / (2 * h)
            d2 = (f(h / 2) - f(-h / 2)) / h
            if abs(d1 - d2) > 1e-3 * max(abs(d1), abs(d2), 1e-9):
                continue  # an L1 sign or a support edge lies within h: a kink
            assert abs(G[i] - d1) <= 1e-5 * abs(d1) + 1e-8, (k, i, G[i], d1)
            checked += 1
    assert checked >= 15


def test_chain_rule_through_loss_images(scene):
    """Gradient of sum_v L_v == the weighted gradient with w = dL_v/dimage_v."""
    w, P = scene
    cams, poses, targets = _args(w, [0, 1, 2])
    L, g, outs = R.multiview_gradients(P, 1, cams, poses, targets)
    wc, wd = [], []
    for out, (trgb, tdep) in zip(outs, targets):
        _, gc, gd = R.loss_image_grads(out["color"].detach(), out["depth"].detach(), trgb, tdep)
        wc.append(gc.numpy())
        wd.append(gd.numpy())
    gw = R.multiview_weighted_gradients(P, 1, cams, poses, wc, wd)
    for k in R.PARAM_NAMES + ("pose",):
        _close(gw[k].numpy(), g[k].numpy(), 1e-10)
