"""Adam update of the Gaussian parameters, float64 (test infrastructure).

The paper optimises the Gaussian parameters "using the gradient descent
method" without naming the optimiser (Sec. III-B.3).  Reading used here:
Adam with bias correction, applied densely to every parameter,

    m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
    p <- p - lr_group * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),

with one learning rate per parameter group.  Pinned against
``torch.optim.Adam`` (a library implementation) in ``tests/test_oracle_adam.py``.

Flat parameter layout for N Gaussians with K = (degree + 1)^2 SH coefficients
per channel, N * (11 + 3K) floats in this order:
    means [N, 3] | log_scales [N, 3] | quats [N, 4] | opacity_logits [N] | sh [N, K, 3]
The SH block's first three floats of every Gaussian (k = 0) form the
"sh_dc" group, the remaining 3(K - 1) the "sh_rest" group.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class AdamCfg:
    lr_means: float = 1.6e-4
    lr_log_scales: float = 5e-3
    lr_quats: float = 1e-3
    lr_opacity: float = 5e-2
    lr_sh_dc: float = 2.5e-3
    lr_sh_rest: float = 1.25e-4
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15


def flat_size(n: int, sh_degree: int) -> int:
    K = (sh_degree + 1) ** 2
    return n * (11 + 3 * K)


def lr_per_element(n: int, sh_degree: int, cfg: AdamCfg) -> np.ndarray:
    K = (sh_degree + 1) ** 2
    sh = np.full((n, K, 3), cfg.lr_sh_rest)
    sh[:, 0, :] = cfg.lr_sh_dc
    return np.concatenate([
        np.full(3 * n, cfg.lr_means), np.full(3 * n, cfg.lr_log_scales), np.full(4 * n, cfg.lr_quats),
        np.full(n, cfg.lr_opacity), sh.ravel(),
    ])


def flatten(params: dict) -> np.ndarray:
    return np.concatenate([np.asarray(params[k], np.float64).ravel()
                           for k in ("means", "log_scales", "quats", "opacity_logits", "sh")])


def adam_step(p, g, m, v, step: int, lr, cfg: AdamCfg):
    """One Adam step (``step`` counts from 1).  Returns new (p, m, v)."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = cfg.beta1 * np.asarray(m, np.float64) + (1.0 - cfg.beta1) * g
    v = cfg.beta2 * np.asarray(v, np.float64) + (1.0 - cfg.beta2) * g * g
    mhat = m / (1.0 - cfg.beta1 ** step)
    vhat = v / (1.0 - cfg.beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + cfg.eps), m, v
