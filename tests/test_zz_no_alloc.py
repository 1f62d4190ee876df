"""gs_loss_l1_noalloc, the loss entry point for callers that must not
allocate device memory (their GPU memory belongs to their own pool, or their
loop cannot absorb an allocation), gives the same loss and image gradients as
gs_loss_l1 on two calls in a row, and rejects images over its size limit.

This file is collected last on purpose: it must pass in a fresh process
(where its first call sets up the fixed scratch array on the device) and
after every other test."""
import numpy as np
import pytest
import torch

from tests._util import ensure_built

pytestmark = pytest.mark.gpu


def _inputs(rng, H, W):
    col = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    dep = rng.uniform(0.5, 4, (H, W)).astype(np.float32)
    trgb = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    tdep = rng.uniform(0.5, 4, (H, W)).astype(np.float32)
    tdep[rng.uniform(0, 1, (H, W)) < 0.1] = 0.0
    return [torch.as_tensor(a, device="cuda") for a in (col, dep, trgb, tdep)]


def _outputs(H, W):
    return torch.zeros(1, device="cuda"), torch.empty((3, H, W), device="cuda"), torch.empty((H, W), device="cuda")


def test_noalloc_loss_matches_context_loss_on_two_calls():
    ensure_built()
    from paper_2408_12677_gb300 import abi
    from paper_2408_12677_gb300.torch_api import Context
    ctx = Context(0)
    rng = np.random.default_rng(2024)
    # two calls in a row with different sizes: the second reuses the array the first filled
    for H, W in ((680, 1200), (48, 64)):
        col, dep, trgb, tdep = _inputs(rng, H, W)
        cam = abi.make_camera(1, 1, 0, 0, W, H)
        L0, gc0, gd0 = _outputs(H, W)
        L1, gc1, gd1 = _outputs(H, W)
        abi.gs_loss_l1(ctx.handle, cam, col, dep, trgb, tdep, 0.8, 0.2, L0, gc0, gd0)
        abi.gs_loss_l1_noalloc(cam, col, dep, trgb, tdep, 0.8, 0.2, L1, gc1, gd1)
        torch.cuda.synchronize()
        assert abs(float(L1) - float(L0)) <= 1e-5 * abs(float(L0))
        np.testing.assert_allclose(gc1.cpu().numpy(), gc0.cpu().numpy(), rtol=1e-6, atol=0)
        np.testing.assert_allclose(gd1.cpu().numpy(), gd0.cpu().numpy(), rtol=1e-6, atol=0)
    ctx.close()


def test_noalloc_loss_rejects_images_over_the_limit():
    ensure_built()
    from paper_2408_12677_gb300 import abi
    lib = abi.load()
    import ctypes as C
    too_big = abi.make_camera(1, 1, 0, 0, 4097, 4096)
    dummy = torch.zeros(1, device="cuda")
    p = dummy.data_ptr()
    st = lib.gs_loss_l1_noalloc(C.byref(too_big), p, p, p, p, 0.8, 0.2, p, p, p, None)
    assert st == 3  # GS_ERR_CAPACITY, nothing enqueued
