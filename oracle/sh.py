"""Real spherical harmonics up to degree 3 (view-dependent colour, Sec. III-A.2).

The paper stores "spherical harmonics (SH) coefficients to capture the
view-dependent color" without fixing a basis.  Reading used here: the real
orthonormal basis obtained from the complex harmonics Y_l^m that include the
Condon-Shortley phase,

    Y_{l,m}  = sqrt(2) Re Y_l^m      (m > 0)
    Y_{l,0}  = Y_l^0
    Y_{l,-m} = sqrt(2) Im Y_l^m      (m > 0)

ordered by k = l^2 + l + m.  With the associated Legendre function written as
P_l^m(z) = (-1)^m (1 - z^2)^{m/2} d^m P_l / dz^m and, for a unit vector
(x, y, z), sin^m(theta) e^{i m phi} = (x + i y)^m, this is

    Y_{l,+-m}(x, y, z) = N_lm (-1)^m (d^m P_l/dz^m)(z) * {Re, Im}(x + i y)^m,
    N_lm = sqrt(2 - [m == 0]) * sqrt((2l + 1)/(4 pi) * (l - m)! / (l + m)!).

The Legendre derivatives come from numpy's Legendre series; nothing here is a
hand-typed table.  Pinned in ``tests/test_oracle_sh.py`` against
``scipy.special`` and by quadrature orthonormality on the sphere.
"""
from __future__ import annotations

import math

import numpy as np
import torch
from numpy.polynomial import legendre as npleg


def _legendre_derivative_power_coeffs(l: int, m: int) -> np.ndarray:
    """Power-series coefficients (ascending) of d^m P_l(z) / dz^m."""
    c = np.zeros(l + 1)
    c[l] = 1.0
    d = npleg.legder(c, m) if m > 0 else c
    return npleg.leg2poly(d) if d.size else np.zeros(1)


def _norm(l: int, m: int) -> float:
    k = math.sqrt((2 * l + 1) / (4.0 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
    return k * (math.sqrt(2.0) if m > 0 else 1.0)


def n_coeffs(degree: int) -> int:
    return (degree + 1) ** 2


def sh_basis(dirs: torch.Tensor, degree: int) -> torch.Tensor:
    """Evaluate the real SH basis at unit vectors ``dirs`` [n, 3] -> [n, (degree+1)^2]."""
    x, y, z = dirs.unbind(-1)
    # (x + i y)^m = re[m] + i im[m]
    re = [torch.ones_like(x)]
    im = [torch.zeros_like(x)]
    for _ in range(degree):
        r, s = re[-1], im[-1]
        re.append(r * x - s * y)
        im.append(s * x + r * y)
    cols = [None] * n_coeffs(degree)
    for l in range(degree + 1):
        for m in range(0, l + 1):
            coeffs = _legendre_derivative_power_coeffs(l, m)
            poly = torch.zeros_like(z)
            for p in range(len(coeffs) - 1, -1, -1):  # Horner
                poly = poly * z + float(coeffs[p])
            base = _norm(l, m) * ((-1.0) ** m) * poly
            if m == 0:
                cols[l * l + l] = base
            else:
                cols[l * l + l + m] = base * re[m]
                cols[l * l + l - m] = base * im[m]
    return torch.stack(cols, -1)


def sh_to_rgb(sh: torch.Tensor, dirs: torch.Tensor, degree: int) -> torch.Tensor:
    """Decoded colour max(0, 0.5 + sum_k Y_k(d) k_k) for sh [n, K, 3]."""
    Y = sh_basis(dirs, degree)
    return torch.clamp_min(0.5 + torch.einsum("nk,nkc->nc", Y, sh), 0.0)


__all__ = ["sh_basis", "sh_to_rgb", "n_coeffs"]
