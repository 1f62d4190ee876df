"""Pins for the oracle's compositing (Eq. 11) and loss (Eq. 12): closed-form
single-Gaussian images, the opaque-front and early-stop rules, invariants,
and brute vs prefilter mode."""
import math

import numpy as np
import pytest
import torch

from oracle import render as R
from synth import workloads
from synth.scene import Camera, look_at

Y00 = 0.5 / math.sqrt(math.pi)
CAM = Camera(60.0, 60.0, 32.0, 24.0, 64, 48)
IDENT = (np.eye(3), np.zeros(3))


def _scene(means, log_scales, logits, colors, quats=None):
    n = len(means)
    sh = ((np.asarray(colors, float) - 0.5) / Y00)[:, None, :]
    if quats is None:
        quats = [[1.0, 0, 0, 0]] * n
    return {"means": np.asarray(means, float), "log_scales": np.asarray(log_scales, float),
            "quats": np.asarray(quats, float), "opacity_logits": np.asarray(logits, float), "sh": sh}


def _render(params, cam=CAM, pose=IDENT, deg=0, **kw):
    return R.render(R.to_tensors(params), deg, cam, *pose, **kw)


@pytest.mark.parametrize("z,s,logit", [(2.0, 0.02, 0.0), (1.0, 0.05, 1.5), (3.0, 0.01, -2.0)])
def test_single_isotropic_gaussian_closed_form(z, s, logit):
    """Pixel value = c * min(0.99, sigmoid(o) exp(-|u - mu|^2 / (2 sigma^2))) where
    the 3-sigma and 1/255 rules allow, sigma^2 = (f s / z)^2 + 0.3."""
    c = np.array([0.9, 0.4, 0.2])
    out = _render(_scene([[0, 0, z]], [[np.log(s)] * 3], [logit], [c]))
    sig2 = (CAM.fx * s / z) ** 2 + 0.3
    jj, ii = np.meshgrid(np.arange(48) + 0.5, np.arange(64) + 0.5, indexing="ij")
    r2 = (ii - 32.0) ** 2 + (jj - 24.0) ** 2
    q = r2 / sig2
    a = np.minimum(0.99, 1 / (1 + math.exp(-logit)) * np.exp(-0.5 * q))
    a = np.where((q <= 9) & (a >= 1 / 255), a, 0.0)
    np.testing.assert_allclose(out["color"].numpy(), c[:, None, None] * a[None], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(out["depth"].numpy(), z * a, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(out["alpha"].numpy(), a, rtol=1e-12, atol=1e-15)
    # four pixels around the centre share the peak exp(-0.25 / sigma^2)
    peak = min(0.99, 1 / (1 + math.exp(-logit)) * math.exp(-0.25 / sig2))
    np.testing.assert_allclose(out["alpha"].numpy()[23:25, 31:33], peak, rtol=1e-12)


def test_pixel_centre_convention():
    """A Gaussian whose mean sits exactly on the centre of pixel (10, 7) gives
    that pixel G = 1, i.e. alpha = min(0.99, opacity)."""
    z = 2.0
    x = (10.5 - CAM.cx) * z / CAM.fx
    y = (7.5 - CAM.cy) * z / CAM.fy
    out = _render(_scene([[x, y, z]], [[np.log(0.01)] * 3], [0.0], [[1, 1, 1]]))
    assert abs(out["alpha"].numpy()[7, 10] - 0.5) < 1e-12
    assert out["alpha"].numpy()[7, 10] == out["alpha"].numpy().max()


def test_opaque_front_hides_all_but_one_percent():
    """A front Gaussian clamped at alpha 0.99 over the whole image lets exactly
    1% of the rest through: image = 0.99 c_front + 0.01 * (render of the rest)."""
    rest = workloads.tiny_random(seed=5, n=60).params
    front = _scene([[0, 0, 0.3]], [[np.log(5.0)] * 3], [20.0], [[0.2, 0.7, 0.4]])
    both = {k: np.concatenate([front[k], np.asarray(rest[k], float)]) for k in front}
    a = _render(both)
    b = _render({k: np.asarray(rest[k], float) for k in front})
    expect = 0.99 * np.array([0.2, 0.7, 0.4])[:, None, None] + 0.01 * b["color"].numpy()
    np.testing.assert_allclose(a["color"].numpy(), expect, rtol=1e-12, atol=1e-15)


def test_three_opaque_fronts_stop_compositing():
    """Two alpha-0.99 layers leave T = 1e-4; the third would push T to 1e-6 <
    1e-4, so it and everything behind contribute exactly nothing."""
    cols = [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]]
    sc = _scene([[0, 0, 0.3], [0, 0, 0.4], [0, 0, 0.5], [0, 0, 0.6]], [[np.log(5.0)] * 3] * 4, [20.0] * 4, cols)
    out = _render(sc)
    img = out["color"].numpy()
    np.testing.assert_allclose(img[:, 10, 10], [0.99, 0.01 * 0.99, 0.0], rtol=1e-12, atol=1e-15)
    assert (out["n_contrib"].numpy() == 2).all()
    np.testing.assert_allclose(out["T_final"].numpy(), 0.01 * 0.01, rtol=1e-9)


def test_invisible_gaussian_below_alpha_min():
    """sigmoid(logit) < 1/255 everywhere: the Gaussian never takes part."""
    out = _render(_scene([[0, 0, 1.0]], [[np.log(0.1)] * 3], [-6.0], [[1, 1, 1]]))
    assert float(out["alpha"].abs().max()) == 0.0


def test_invariants_random_scene():
    w = workloads.tiny_random(seed=11, n=300)
    out = _render({k: np.asarray(w.params[k], float) for k in R.PARAM_NAMES})
    T = out["T_final"].numpy()
    assert (T >= 0).all() and (T <= 1).all()
    a = out["alpha"].numpy()
    assert (a >= 0).all() and (a < 1).all()
    cmax = out["proj"]["rgb"].detach().numpy().max()
    assert out["color"].numpy().max() <= cmax + 1e-12


def test_permutation_invariance():
    w = workloads.tiny_random(seed=12, n=200)
    P = {k: np.asarray(w.params[k], float) for k in R.PARAM_NAMES}
    perm = np.random.default_rng(0).permutation(200)
    Q = {k: v[perm] for k, v in P.items()}
    a, b = _render(P), _render(Q)
    np.testing.assert_allclose(a["color"].numpy(), b["color"].numpy(), rtol=0, atol=1e-15)


def test_rigid_motion_invariance(rng):
    """Moving the map and the camera by the same rigid motion changes nothing
    (SH degree 3, so the view direction is exercised too)."""
    w = workloads.tiny_random(seed=13, n=150, sh_degree=3, sh_rest_std=0.1)
    P = {k: np.asarray(w.params[k], float) for k in R.PARAM_NAMES}
    from scipy.spatial.transform import Rotation
    G = Rotation.from_rotvec([0.3, -0.5, 0.8]).as_matrix()
    tr = np.array([1.0, -2.0, 0.5])
    Q = dict(P)
    Q["means"] = P["means"] @ G.T + tr
    # rotate each Gaussian's frame: q' = g * q
    gq = Rotation.from_matrix(G).as_quat()[[3, 0, 1, 2]]
    w0, x0, y0, z0 = gq
    qs = P["quats"]
    Q["quats"] = np.stack([
        w0 * qs[:, 0] - x0 * qs[:, 1] - y0 * qs[:, 2] - z0 * qs[:, 3],
        w0 * qs[:, 1] + x0 * qs[:, 0] + y0 * qs[:, 3] - z0 * qs[:, 2],
        w0 * qs[:, 2] - x0 * qs[:, 3] + y0 * qs[:, 0] + z0 * qs[:, 1],
        w0 * qs[:, 3] + x0 * qs[:, 2] - y0 * qs[:, 1] + z0 * qs[:, 0]], 1)
    # SH coefficients are expressed in the world frame: rotating the world
    # rotates the colour field, so compare the view-independent (deg-0) part
    # with a pose moved accordingly.  T_CW' = T_CW G^-1.
    Rc, tc = np.eye(3), np.zeros(3)
    Rc2 = Rc @ G.T
    tc2 = tc - Rc2 @ tr
    P0 = dict(P, sh=P["sh"][:, :1])
    Q0 = dict(Q, sh=Q["sh"][:, :1])
    a = _render(P0)
    b = _render(Q0, pose=(Rc2, tc2))
    np.testing.assert_allclose(a["color"].numpy(), b["color"].numpy(), atol=1e-11)
    np.testing.assert_allclose(a["depth"].numpy(), b["depth"].numpy(), atol=1e-11)
    # translation only: the full SH colour is invariant too
    Qt = dict(P, means=P["means"] + tr)
    c = _render(P, deg=3)
    d = _render(Qt, pose=(Rc, tc - tr), deg=3)
    np.testing.assert_allclose(c["color"].numpy(), d["color"].numpy(), atol=1e-11)


def test_brute_equals_prefilter():
    """Dropping Gaussians with q > 9 at every pixel of a chunk changes nothing:
    identical blend sets, values equal up to the summation order (1e-13)."""
    w = workloads.tiny_random(seed=14, n=400, sh_degree=1, sh_rest_std=0.1)
    P = {k: np.asarray(w.params[k], float) for k in R.PARAM_NAMES}
    a = _render(P, deg=1, prefilter=False)
    b = _render(P, deg=1, prefilter=True)
    assert torch.equal(a["n_contrib"], b["n_contrib"])
    for k in ("color", "depth", "alpha"):
        np.testing.assert_allclose(a[k].numpy(), b[k].numpy(), rtol=1e-13, atol=1e-15, err_msg=k)


def test_pixel_subset_matches_full_image(rng):
    w = workloads.tiny_random(seed=15, n=300)
    P = {k: np.asarray(w.params[k], float) for k in R.PARAM_NAMES}
    full = _render(P)
    pix = np.stack([rng.integers(0, 64, 50), rng.integers(0, 48, 50)], 1)
    sub = _render(P, pixels=pix, prefilter=True)
    np.testing.assert_allclose(sub["color"].numpy(), full["color"].numpy()[:, pix[:, 1], pix[:, 0]], rtol=1e-13)
    np.testing.assert_allclose(sub["depth"].numpy(), full["depth"].numpy()[pix[:, 1], pix[:, 0]], rtol=1e-13)
    np.testing.assert_array_equal(sub["n_contrib"].numpy(), full["n_contrib"].numpy()[pix[:, 1], pix[:, 0]])


def test_loss_closed_form():
    H, W = 4, 5
    tgt = np.full((3, H, W), 0.5)
    tdep = np.full((H, W), 2.0)
    tdep[0, :] = 0.0  # invalid target depth is ignored
    col = torch.as_tensor(tgt + 0.1)
    dep = torch.as_tensor(tdep + 0.3)
    L = float(R.loss_l1(col, dep, tgt, tdep))
    assert abs(L - (0.8 * 0.1 + 0.2 * 0.3)) < 1e-12
    _, gc, gd = R.loss_image_grads(tgt + 0.1, tdep + 0.3, tgt, tdep)
    np.testing.assert_allclose(gc.numpy(), 0.8 / (3 * H * W))
    expect = np.full((H, W), 0.2 / (H * W - W))
    expect[0, :] = 0.0
    np.testing.assert_allclose(gd.numpy(), expect)
    _, gc0, _ = R.loss_image_grads(tgt, tdep, tgt, tdep)
    assert float(gc0.abs().max()) == 0.0  # sign(0) = 0


def test_brute_equals_bbox_prefilter_on_tiles():
    """The bounding-box selection per tile keeps every Gaussian with q <= 9 at
    a pixel of the tile: same blend sets and values as brute force, over all
    tiles of a ragged image in a permuted tile order."""
    w = workloads.tiny_random(seed=16, n=500, sh_degree=1, sh_rest_std=0.1)
    P = {k: np.asarray(w.params[k], float) for k in R.PARAM_NAMES}
    full = _render(P, deg=1, prefilter=False)
    tiles = np.random.default_rng(3).permutation(4 * 3)  # 64 x 48 in 16 x 16 tiles
    pix = R.tile_pixels(CAM, tiles)
    sub = _render(P, deg=1, pixels=pix, prefilter="bbox", chunk_px=256)
    # ragged tiles (70 x 50 in 16 x 16: 6- and 2-pixel edges) grouped by tile
    cam = Camera(60.0, 60.0, 35.0, 25.0, 70, 50)
    full2 = _render(P, cam=cam, deg=1, prefilter=False)
    pix2, sizes = R.tile_pixels(cam, np.random.default_rng(4).permutation(5 * 4), sizes=True)
    sub2 = _render(P, cam=cam, deg=1, pixels=pix2, prefilter="bbox", chunk_px=sizes)
    np.testing.assert_array_equal(sub2["n_contrib"].numpy(), full2["n_contrib"].numpy()[pix2[:, 1], pix2[:, 0]])
    np.testing.assert_allclose(sub2["color"].numpy(), full2["color"].numpy()[:, pix2[:, 1], pix2[:, 0]],
                               rtol=1e-13, atol=1e-15)
    np.testing.assert_array_equal(sub["n_contrib"].numpy(), full["n_contrib"].numpy()[pix[:, 1], pix[:, 0]])
    np.testing.assert_allclose(sub["color"].numpy(), full["color"].numpy()[:, pix[:, 1], pix[:, 0]], rtol=1e-13,
                               atol=1e-15)
    np.testing.assert_allclose(sub["alpha"].numpy(), full["alpha"].numpy()[pix[:, 1], pix[:, 0]], rtol=1e-13,
                               atol=1e-15)
    # a ragged tile at the image corner is clipped to the image
    cam = Camera(60.0, 60.0, 32.0, 24.0, 70, 50)
    p2 = R.tile_pixels(cam, [3 * 5 + 4])  # last tile of 5 x 4: 6 x 2 pixels
    assert p2.shape == (12, 2) and p2[:, 0].min() == 64 and p2[:, 1].min() == 48


def test_decision_margins_single_gaussian():
    """One isotropic Gaussian: the q margin of a pixel is |q - 9| / 9 with q the
    closed-form |u - mu|^2 / sigma^2, its alpha margins are the distances of
    sigmoid(o) exp(-q/2) to 1/255 and 0.99, and a lone Gaussian never meets
    the stop rule (T (1 - alpha) >= 0.01)."""
    z, s, logit = 2.0, 0.02, 0.0
    out = R.decision_margins(_scene([[0, 0, z]], [[np.log(s)] * 3], [logit], [[0.5, 0.5, 0.5]]), 0, CAM, *IDENT)
    sig2 = (CAM.fx * s / z) ** 2 + 0.3
    jj, ii = np.meshgrid(np.arange(48) + 0.5, np.arange(64) + 0.5, indexing="ij")
    q = (((ii - 32.0) ** 2 + (jj - 24.0) ** 2) / sig2).ravel()
    a = 0.5 * np.exp(-0.5 * q)
    want = np.where(q <= 9 * (1 + 1e-3), np.abs(q - 9) / 9, np.inf)
    want = np.minimum(want, np.where(q <= 9, np.abs(a - 1 / 255) * 255, np.inf))
    want = np.minimum(want, np.where(q <= 9, np.abs(a - 0.99) / 0.99, np.inf))
    want = np.minimum(want, np.where((q <= 9) & (a >= 1 / 255), np.abs((1 - a) - 1e-4) / 1e-4, np.inf))
    np.testing.assert_allclose(out["pixel"], want, rtol=1e-9)
    assert out["gauss"][0] == pytest.approx(want.min(), rel=1e-9)


def test_decision_margins_stop_rule():
    """Three opaque fronts (alpha = 0.99 each) over one pixel: before the
    second, T = 0.01, so its stop test T (1 - alpha) = 1e-4 lies exactly on
    the threshold (distance 0: a float32 evaluation may take it either way);
    with the middle front half as opaque the nearest decision is the clamp of
    the others instead."""
    P = _scene([[0, 0, 1.0], [0, 0, 1.5], [0, 0, 2.0]], [[np.log(0.5)] * 3] * 3, [20.0] * 3, [[0.5] * 3] * 3)
    out = R.decision_margins(P, 0, CAM, *IDENT, pixels=np.array([[32, 24]]))
    assert out["pixel"][0] < 1e-12
    assert R.MARGIN_KINDS[out["pixel_kind"][0]] == "T (1 - alpha) = 1e-4"
    P["opacity_logits"][1] = 0.0  # alpha 0.5: the stop tests are now far (T (1 - alpha) = 0.005, 5e-5)
    out = R.decision_margins(P, 0, CAM, *IDENT, pixels=np.array([[32, 24]]))
    sigmoid20 = 1 / (1 + np.exp(-20.0))
    want = []
    for z in (1.0, 2.0):  # the two opaque fronts: q = |(0.5, 0.5)|^2 / sigma^2 at the pixel centre
        q = 0.5 / ((CAM.fx * 0.5 / z) ** 2 + 0.3)
        want.append(abs(sigmoid20 * np.exp(-0.5 * q) - 0.99) / 0.99)
    assert out["pixel"][0] == pytest.approx(min(want), rel=1e-6)
    assert R.MARGIN_KINDS[out["pixel_kind"][0]] == "alpha = 0.99"


def test_decision_margins_bbox_equals_brute():
    """Margins computed tile by tile with the bounding-box selection equal
    the brute-force ones (a dropped Gaussian has no decision near a
    threshold at any pixel of the tile)."""
    w = workloads.tiny_random(seed=17, n=400)
    P = {k: np.asarray(w.params[k], float) for k in R.PARAM_NAMES}
    a = R.decision_margins(P, 0, CAM, *IDENT)
    pix, sizes = R.tile_pixels(CAM, range(12), sizes=True)
    b = R.decision_margins(P, 0, CAM, *IDENT, pixels=pix, prefilter="bbox", chunk_px=sizes)
    lin = pix[:, 1] * CAM.width + pix[:, 0]
    np.testing.assert_array_equal(a["pixel"][lin], b["pixel"])
    np.testing.assert_array_equal(a["pixel_kind"][lin], b["pixel_kind"])
    np.testing.assert_array_equal(a["gauss"], b["gauss"])
