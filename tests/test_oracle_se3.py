"""Pins for the oracle's pose twist (the left perturbation exp(xi^) T_CW of the
camera pose, xi = (rho, phi), whose gradient the backward pass returns).

The oracle takes exp(xi^) as the matrix exponential of the 4x4 twist matrix.
These tests pin it to what does not depend on that code: the rotation block
against scipy's rotation-vector map, the translation against the closed-form
SE(3) left Jacobian V(phi) rho (Rodrigues' formulas), the group law of
one-parameter subgroups, and the left-perturbation convention on a known
point (the perturbation acts on camera-frame coordinates, after T_CW).  A
sign or transpose slip in the skew matrix, a right instead of a left
perturbation, or rho and phi swapped each fail one of them."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from oracle import render as R

DT = torch.float64


def _skew(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def _closed_form(rho, phi):
    """Rotation (scipy) and V(phi) rho (Rodrigues' left Jacobian of SO(3))."""
    th = np.linalg.norm(phi)
    K = _skew(phi)
    if th < 1e-8:
        V = np.eye(3) + 0.5 * K
    else:
        V = np.eye(3) + (1 - np.cos(th)) / th ** 2 * K + (th - np.sin(th)) / th ** 3 * (K @ K)
    return Rotation.from_rotvec(phi).as_matrix(), V @ rho


TWISTS = [
    ([0.1, -0.2, 0.3], [0.0, 0.0, 0.0]),
    ([0.0, 0.0, 0.0], [0.0, 0.0, 0.7]),
    ([0.3, 0.1, -0.4], [0.2, -0.5, 0.1]),
    ([-1.0, 0.5, 2.0], [1.1, 0.4, -0.9]),
    ([0.02, 0.01, -0.03], [1e-4, -2e-4, 3e-4]),
    ([0.5, -0.5, 0.25], [-2.5, 0.3, 0.8]),
]


def _check_exp(se3_exp, rho, phi):
    rho, phi = np.asarray(rho, np.float64), np.asarray(phi, np.float64)
    E = se3_exp(torch.as_tensor(np.concatenate([rho, phi]), dtype=DT)).numpy()
    Rr, tr = _closed_form(rho, phi)
    np.testing.assert_allclose(E[:3, :3], Rr, atol=1e-12)
    np.testing.assert_allclose(E[:3, 3], tr, atol=1e-12)
    np.testing.assert_allclose(E[3], [0, 0, 0, 1], atol=1e-15)


@pytest.mark.parametrize("rho,phi", TWISTS)
def test_se3_exp_matches_rotvec_and_left_jacobian(rho, phi):
    _check_exp(R.se3_exp, rho, phi)


def test_se3_exp_rotation_about_z_is_counterclockwise():
    th = 0.3
    E = R.se3_exp(torch.tensor([0, 0, 0, 0, 0, th], dtype=DT)).numpy()
    np.testing.assert_allclose(E[:3, :3], [[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]],
                               atol=1e-14)


def test_se3_exp_one_parameter_subgroup():
    xi = torch.tensor([0.3, -0.2, 0.5, 0.4, 0.1, -0.6], dtype=DT)
    E1 = R.se3_exp(xi)
    E2 = R.se3_exp(2 * xi)
    np.testing.assert_allclose((E1 @ E1).numpy(), E2.numpy(), atol=1e-12)
    np.testing.assert_allclose((E1 @ R.se3_exp(-xi)).numpy(), np.eye(4), atol=1e-12)


@pytest.mark.parametrize("rho,phi", TWISTS[2:])
def test_perturb_pose_is_a_left_perturbation_on_a_known_point(rho, phi):
    rng = np.random.default_rng(5)
    R_cw = Rotation.from_rotvec(rng.normal(size=3)).as_matrix()
    t_cw = rng.normal(size=3)
    p_w = np.array([0.7, -1.2, 3.4])
    Rp, tp = R.perturb_pose(torch.as_tensor(R_cw, dtype=DT), torch.as_tensor(t_cw, dtype=DT),
                            torch.as_tensor(np.concatenate([rho, phi]), dtype=DT))
    got = Rp.numpy() @ p_w + tp.numpy()
    Rr, tr = _closed_form(np.asarray(rho), np.asarray(phi))
    p_c = R_cw @ p_w + t_cw
    np.testing.assert_allclose(got, Rr @ p_c + tr, atol=1e-12)
    # a right perturbation T_CW exp(xi^) moves the point differently
    right = R_cw @ (Rr @ p_w + tr) + t_cw
    assert np.linalg.norm(got - right) > 1e-3


def _planted_transposed_skew(xi):
    """The twist matrix with its rotation block transposed (a plausible slip)."""
    rho, phi = xi[:3], xi[3:]
    z = torch.zeros((), dtype=xi.dtype)
    A = torch.stack([
        torch.stack([z, phi[2], -phi[1], rho[0]]),
        torch.stack([-phi[2], z, phi[0], rho[1]]),
        torch.stack([phi[1], -phi[0], z, rho[2]]),
        torch.stack([z, z, z, z]),
    ])
    return torch.linalg.matrix_exp(A)


def _planted_swapped(xi):
    """rho and phi swapped."""
    return R.se3_exp(torch.cat([xi[3:], xi[:3]]))


@pytest.mark.parametrize("planted", [_planted_transposed_skew, _planted_swapped])
def test_planted_mistakes_fail_the_pin(planted):
    with pytest.raises(AssertionError):
        _check_exp(planted, *TWISTS[2])
