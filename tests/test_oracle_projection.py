"""Pins for the oracle's projection (Eq. 2-5): closed forms, a library
rotation, finite-difference Jacobians and Monte Carlo covariances."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from oracle import render as R
from synth.scene import Camera, Pose, look_at

DT = torch.float64


def _P(means, log_scales, quats, logits=None, sh=None):
    n = len(means)
    if logits is None:
        logits = np.zeros(n)
    if sh is None:
        sh = np.zeros((n, 1, 3))
    return R.to_tensors({"means": np.asarray(means, float), "log_scales": np.asarray(log_scales, float),
                         "quats": np.asarray(quats, float), "opacity_logits": np.asarray(logits, float),
                         "sh": np.asarray(sh, float)})


CAM = Camera(600.0, 500.0, 320.0, 240.0, 640, 480)
IDENT = (np.eye(3), np.zeros(3))


def test_quat_matches_scipy_rotation(rng):
    q = rng.standard_normal((64, 4)) * rng.uniform(0.2, 5.0, (64, 1))
    mine = R.quat_to_rotmat(torch.as_tensor(q)).numpy()
    ref = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()  # scipy is scalar-last
    np.testing.assert_allclose(mine, ref, atol=1e-13)
    np.testing.assert_allclose(R.quat_to_rotmat(torch.as_tensor(-q)).numpy(), ref, atol=1e-13)
    eye = np.einsum("nij,nkj->nik", mine, mine)
    np.testing.assert_allclose(eye, np.broadcast_to(np.eye(3), eye.shape), atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(mine), 1.0, atol=1e-13)


def test_covariance_matches_library_rotation(rng):
    q = rng.standard_normal((16, 4))
    ls = rng.uniform(-3, 0, (16, 3))
    Rm = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()
    ref = np.einsum("nij,nj,nkj->nik", Rm, np.exp(2 * ls), Rm)
    mine = R.covariance_3d(torch.as_tensor(ls), torch.as_tensor(q)).numpy()
    np.testing.assert_allclose(mine, ref, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("z,s", [(1.0, 0.01), (2.5, 0.05), (4.0, 0.2)])
def test_isotropic_on_axis_closed_form(z, s, rng):
    """A Gaussian at (0, 0, z) with scale s projects to the principal point with
    covariance diag((fx s/z)^2 + 0.3, (fy s/z)^2 + 0.3), whatever its rotation."""
    P = _P([[0.0, 0.0, z]], [[np.log(s)] * 3], [rng.standard_normal(4)])
    pr = R.project(P, 0, CAM, *IDENT)
    np.testing.assert_allclose(pr["mean2d"].numpy()[0], [CAM.cx, CAM.cy], atol=1e-12)
    cov = np.diag([(CAM.fx * s / z) ** 2 + 0.3, (CAM.fy * s / z) ** 2 + 0.3])
    np.testing.assert_allclose(pr["cov2d"].numpy()[0], cov, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(pr["conic"].numpy()[0], [1 / cov[0, 0], 0.0, 1 / cov[1, 1]], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(pr["depth"].numpy()[0], z)


def _pi(pc):
    return np.array([CAM.fx * pc[0] / pc[2] + CAM.cx, CAM.fy * pc[1] / pc[2] + CAM.cy])


def test_cov2d_is_fd_jacobian_of_pi_along_the_major_axis(rng):
    """For a needle-shaped Gaussian (scales s, e, e with e << s) the 2D
    covariance minus the 0.3 dilation is s^2 v v^T with v the directional
    derivative of the projection along the needle, W R e_x; v is taken by
    central differences and R from scipy."""
    pose = look_at([0.3, -0.2, 0.1], [1.0, 2.0, 0.5])
    W = pose.R.astype(float)
    t = pose.t.astype(float)
    for _ in range(8):
        q = rng.standard_normal(4)
        Rm = Rotation.from_quat(q[[1, 2, 3, 0]]).as_matrix()
        pc = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.4, 0.4), rng.uniform(1.0, 3.0)])
        p = np.linalg.solve(W, pc - t)
        s, e = 0.05, 1e-9
        P = _P([p], [[np.log(s), np.log(e), np.log(e)]], [q])
        pr = R.project(P, 0, CAM, W, t)
        d = W @ Rm[:, 0]
        h = 1e-6
        v = (_pi(pc + h * d) - _pi(pc - h * d)) / (2 * h)
        got = pr["cov2d"].numpy()[0] - 0.3 * np.eye(2)
        np.testing.assert_allclose(got, s * s * np.outer(v, v), rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(pr["mean2d"].numpy()[0], _pi(pc), rtol=1e-12)


def test_cov2d_monte_carlo(rng):
    """Sample covariance of projected 3D samples of a small Gaussian equals
    the EWA covariance (first-order, so only up to O(sigma/z))."""
    q = rng.standard_normal(4)
    ls = np.log([0.004, 0.002, 0.001])
    Rm = Rotation.from_quat(q[[1, 2, 3, 0]]).as_matrix()
    Sig = Rm @ np.diag(np.exp(2 * ls)) @ Rm.T
    p = np.array([0.2, -0.1, 1.5])
    x = rng.multivariate_normal(p, Sig, 400_000)
    uv = np.stack([CAM.fx * x[:, 0] / x[:, 2] + CAM.cx, CAM.fy * x[:, 1] / x[:, 2] + CAM.cy], 1)
    emp = np.cov(uv.T)
    pr = R.project(_P([p], [ls], [q]), 0, CAM, *IDENT)
    got = pr["cov2d"].numpy()[0] - 0.3 * np.eye(2)
    np.testing.assert_allclose(got, emp, rtol=2e-2, atol=2e-2 * np.abs(emp).max())


def test_pose_convention_look_at():
    """A camera looking at a target puts it at the principal point, at depth
    equal to the distance; the camera centre is -R^T t."""
    eye, target = np.array([1.0, 2.0, 1.5]), np.array([4.0, 3.0, 1.0])
    pose = look_at(eye, target)
    P = _P([target], [[-3.0] * 3], [[1, 0, 0, 0]])
    pr = R.project(P, 0, CAM, pose.R.astype(float), pose.t.astype(float))
    np.testing.assert_allclose(pr["mean2d"].numpy()[0], [CAM.cx, CAM.cy], atol=1e-4)
    np.testing.assert_allclose(pr["depth"].numpy()[0], np.linalg.norm(target - eye), rtol=1e-6)
    np.testing.assert_allclose(pose.center, eye, atol=1e-5)


def test_near_plane_culling():
    P = _P([[0, 0, 0.1], [0, 0, 0.2], [0, 0, 0.2001], [0, 0, -1.0]], [[-3.0] * 3] * 4, [[1, 0, 0, 0]] * 4)
    pr = R.project(P, 0, CAM, *IDENT)
    assert pr["idx"].tolist() == [2]


def test_frustum_clamp_uses_clamped_position(rng):
    """Off-screen beyond 1.3x the half field of view, J is evaluated at the
    clamped ray: the 2D covariance equals that of a Gaussian on the clamp ray."""
    z = 2.0
    lim = 1.3 * CAM.width / (2 * CAM.fx)
    q = rng.standard_normal(4)
    ls = [np.log(0.05), np.log(0.02), np.log(0.01)]
    far = _P([[3.0 * lim * z, 0.1, z]], [ls], [q])
    edge = _P([[lim * z, 0.1, z]], [ls], [q])
    c_far = R.project(far, 0, CAM, *IDENT)["cov2d"].numpy()[0]
    c_edge = R.project(edge, 0, CAM, *IDENT)["cov2d"].numpy()[0]
    np.testing.assert_allclose(c_far, c_edge, rtol=1e-12)
