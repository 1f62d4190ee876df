"""Pins for the oracle Adam update: torch.optim.Adam (a library
implementation) over several steps with per-group learning rates, and the
first-step closed form p1 = p0 - lr g / (|g| + eps)."""
import numpy as np
import torch

from oracle import adam


def test_matches_torch_optim_adam_with_groups(rng):
    n, deg = 37, 3
    cfg = adam.AdamCfg(eps=1e-8)
    size = adam.flat_size(n, deg)
    p0 = rng.standard_normal(size)
    lr = adam.lr_per_element(n, deg, cfg)
    groups = {}
    for v in np.unique(lr):
        groups[v] = np.flatnonzero(lr == v)
    tens = {v: torch.tensor(p0[idx], dtype=torch.float64, requires_grad=True) for v, idx in groups.items()}
    opt = torch.optim.Adam([{"params": [t], "lr": float(v)} for v, t in tens.items()],
                           betas=(cfg.beta1, cfg.beta2), eps=cfg.eps)
    p, m, v2 = p0.copy(), np.zeros(size), np.zeros(size)
    for step in range(1, 6):
        g = rng.standard_normal(size)
        opt.zero_grad()
        for val, t in tens.items():
            t.grad = torch.tensor(g[groups[val]], dtype=torch.float64)
        opt.step()
        p, m, v2 = adam.adam_step(p, g, m, v2, step, lr, cfg)
        ref = np.empty(size)
        for val, t in tens.items():
            ref[groups[val]] = t.detach().numpy()
        np.testing.assert_allclose(p, ref, rtol=1e-13, atol=1e-15)


def test_first_step_closed_form(rng):
    cfg = adam.AdamCfg()
    g = rng.standard_normal(100)
    p0 = rng.standard_normal(100)
    lr = np.full(100, 0.01)
    p1, m1, v1 = adam.adam_step(p0, g, np.zeros(100), np.zeros(100), 1, lr, cfg)
    np.testing.assert_allclose(p1, p0 - 0.01 * g / (np.abs(g) + cfg.eps), rtol=1e-12)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(v1, 0.001 * g * g)


def test_layout_groups():
    n, deg = 3, 1
    cfg = adam.AdamCfg()
    lr = adam.lr_per_element(n, deg, cfg)
    assert lr.size == adam.flat_size(n, deg) == n * (11 + 12)
    assert (lr[:9] == cfg.lr_means).all() and (lr[9:18] == cfg.lr_log_scales).all()
    assert (lr[18:30] == cfg.lr_quats).all() and (lr[30:33] == cfg.lr_opacity).all()
    sh = lr[33:].reshape(n, 4, 3)
    assert (sh[:, 0] == cfg.lr_sh_dc).all() and (sh[:, 1:] == cfg.lr_sh_rest).all()
