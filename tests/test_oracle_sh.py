"""Pins for the real SH basis: scipy's complex harmonics, textbook low-order
closed forms (signs), and quadrature orthonormality on the sphere."""
import math

import numpy as np
import pytest
import scipy.special as sps
import torch

from oracle import sh


def _dirs(rng, n):
    d = rng.standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def _complex_sh(l, m, theta, phi):
    if hasattr(sps, "sph_harm_y"):
        return sps.sph_harm_y(l, m, theta, phi)
    return sps.sph_harm(m, l, phi, theta)  # older scipy: (m, n, azimuth, polar)


def test_matches_scipy_complex_harmonics(rng):
    d = _dirs(rng, 200)
    Y = sh.sh_basis(torch.as_tensor(d), 3).numpy()
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    for l in range(4):
        for m in range(-l, l + 1):
            c = _complex_sh(l, abs(m), theta, phi)
            if m > 0:
                ref = math.sqrt(2) * c.real
            elif m < 0:
                ref = math.sqrt(2) * c.imag
            else:
                ref = c.real
            np.testing.assert_allclose(Y[:, l * l + l + m], ref, atol=1e-12, err_msg=f"l={l} m={m}")


def test_low_order_closed_forms(rng):
    d = _dirs(rng, 50)
    x, y, z = d.T
    Y = sh.sh_basis(torch.as_tensor(d), 2).numpy()
    c0 = 0.5 / math.sqrt(math.pi)
    c1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(Y[:, 0], c0, atol=1e-15)
    np.testing.assert_allclose(Y[:, 1], -c1 * y, atol=1e-14)
    np.testing.assert_allclose(Y[:, 2], c1 * z, atol=1e-14)
    np.testing.assert_allclose(Y[:, 3], -c1 * x, atol=1e-14)
    np.testing.assert_allclose(Y[:, 6], 0.25 * math.sqrt(5 / math.pi) * (3 * z * z - 1), atol=1e-14)
    np.testing.assert_allclose(Y[:, 8], 0.25 * math.sqrt(15 / math.pi) * (x * x - y * y), atol=1e-14)


def test_orthonormal_by_quadrature():
    zs, wz = np.polynomial.legendre.leggauss(12)
    nphi = 16
    phis = np.arange(nphi) * 2 * np.pi / nphi
    Z, PHI = np.meshgrid(zs, phis, indexing="ij")
    W = np.repeat(wz[:, None], nphi, 1) * (2 * np.pi / nphi)
    r = np.sqrt(1 - Z**2)
    d = np.stack([r * np.cos(PHI), r * np.sin(PHI), Z], -1).reshape(-1, 3)
    Y = sh.sh_basis(torch.as_tensor(d), 3).numpy()
    G = Y.T @ (Y * W.reshape(-1, 1))
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_decode_clamps_at_zero(deg, rng):
    K = (deg + 1) ** 2
    coef = torch.as_tensor(rng.normal(0, 1.5, (40, K, 3)))
    d = torch.as_tensor(_dirs(rng, 40))
    rgb = sh.sh_to_rgb(coef, d, deg).numpy()
    raw = 0.5 + np.einsum("nk,nkc->nc", sh.sh_basis(d, deg).numpy(), coef.numpy())
    np.testing.assert_allclose(rgb, np.maximum(raw, 0))
    assert (rgb >= 0).all()
