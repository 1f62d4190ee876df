"""Graph-mode (no-sync) binning into per-tile buckets: while the sync-mode
passes have seen every tile list at most 2048 entries long, no-sync passes
let the projection write every (tile, Gaussian) pair straight into its
tile's bucket (twice the longest list seen, rounded up to a power of two
from 1024 to 4096) and skip the scan and the scatter.  The per-tile lists,
and with them every image, are the same as the counting-scatter binning's
bit for bit; the gradients agree up to the order of the float32 atomics.
Lists that grow past 512 entries take the sort's block-wide path; a list
past its bucket is reported as GS_ERR_CAPACITY and the context goes back to
the counting-scatter binning."""
import numpy as np
import pytest
import torch

from synth import workloads
from synth.scene import Camera, look_at
from tests._util import compare, ensure_built, gpu_render, to_gpu_model
from tests.test_gpu_batched import _batched_render

pytestmark = pytest.mark.gpu


def _scene(seed=3, n=10000, log_scale_range=(-4.5, -2.5)):
    cam = Camera(180.0, 180.0, 96.0, 72.0, 192, 144)
    pose = look_at([0.0, 0.0, 0.0], [2.5, 0.0, 0.0])
    P = workloads.random_gaussians(np.random.default_rng(seed), n, cam, pose, 3, z_range=(1.5, 4.0),
                                   log_scale_range=log_scale_range, sh_rest_std=0.1)
    return P, cam, pose


def _ctx():
    ensure_built()
    from paper_2408_12677_gb300.torch_api import Context
    return Context(0)


def _longest(ctx, cam, tile=16):
    from paper_2408_12677_gb300 import abi
    n_tiles = -(-cam.width // tile) * -(-cam.height // tile)
    r = torch.empty((n_tiles, 2), dtype=torch.int32, device="cuda")
    abi.gs_get_tile_ranges(ctx.handle, r)
    torch.cuda.synchronize()
    r = r.cpu().numpy().view(np.uint32).astype(np.int64)
    return int((r[:, 1] - r[:, 0]).max())


def _length_class(n):
    """Four classes per octave of the list length (0 for an empty list)."""
    n = np.asarray(n, np.int64)
    lead = np.where(n > 0, np.floor(np.log2(np.maximum(n, 1))).astype(np.int64), 0)
    frac = np.where(lead >= 2, (n >> np.maximum(lead - 2, 0)) & 3, (n << np.maximum(2 - lead, 0)) & 3)
    return np.where(n > 0, 4 * lead + frac + 1, 0)


def check_visit_order(ctx, n_tiles):
    """The raster visit order of the last forward pass is a permutation of
    the tiles with non-increasing length classes."""
    from paper_2408_12677_gb300 import abi
    r = torch.empty((n_tiles, 2), dtype=torch.int32, device="cuda")
    o = torch.empty(n_tiles, dtype=torch.int32, device="cuda")
    abi.gs_get_tile_ranges(ctx.handle, r)
    abi.gs_get_tile_order(ctx.handle, o)
    torch.cuda.synchronize()
    r = r.cpu().numpy().view(np.uint32).astype(np.int64)
    o = o.cpu().numpy().view(np.uint32).astype(np.int64)
    np.testing.assert_array_equal(np.sort(o), np.arange(n_tiles))
    cls = _length_class(r[o, 1] - r[o, 0])
    assert (np.diff(cls) <= 0).all()


def test_length_classes():
    assert _length_class([0, 1, 2, 3, 4, 5, 6, 7, 8, 451, 512, 1024]).tolist() == [
        0, 1, 5, 7, 9, 10, 11, 12, 13, 4 * 8 + 3 + 1, 4 * 9 + 1, 4 * 10 + 1]


def _no_sync(ctx, n, npx, pairs):
    from paper_2408_12677_gb300 import abi
    abi.gs_ctx_reserve(ctx.handle, n, npx, pairs)
    abi.gs_ctx_set_sync(ctx.handle, False)


def _launches_of_render(ctx, model, cam, pose):
    before = ctx.stats()["kernel_launches"]
    out = gpu_render(ctx, model, cam, pose)
    return ctx.stats()["kernel_launches"] - before, out


def test_bucket_binning_renders_the_same_images_and_gradients():
    from tests.test_gpu_grad import NAMES
    from tests._util import gpu_backward
    P, cam, pose = _scene()
    ctx = _ctx()
    model = to_gpu_model(P)
    n_sync, ref = _launches_of_render(ctx, model, cam, pose)  # counting-scatter binning
    assert 0 < _longest(ctx, cam) <= 512
    T = -(-cam.width // 16) * -(-cam.height // 16)
    check_visit_order(ctx, T)
    rng = np.random.default_rng(5)
    H, W = cam.height, cam.width
    wc = rng.standard_normal((3, H, W)).astype(np.float32)
    wd = rng.standard_normal((H, W)).astype(np.float32)
    wa = rng.standard_normal((H, W)).astype(np.float32)
    g_ref = gpu_backward(ctx, model, cam, pose, wc, wd, wa)
    _no_sync(ctx, P["means"].shape[0], H * W, 2_000_000)
    n_bucket, got = _launches_of_render(ctx, model, cam, pose)
    assert n_bucket < n_sync  # no count, scan or scatter launch
    check_visit_order(ctx, T)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
    g = gpu_backward(ctx, model, cam, pose, wc, wd, wa)
    for k in NAMES + ("pose",):
        ref_k = g_ref[k]
        compare(k, g[k], ref_k, 1e-5, 1e-6 * np.abs(ref_k).max() + 1e-12, 1e-5)
    from paper_2408_12677_gb300 import abi
    abi.gs_sync_status(ctx.handle)  # no overflow
    ctx.close()


def test_bucket_binning_of_lists_longer_than_a_warp_sorts():
    """The sync pass sees short lists; the Gaussians then grow, so the
    no-sync pass's buckets hold lists of 513-1024 entries (block-wide sort)."""
    P, cam, pose = _scene(seed=4, n=20000, log_scale_range=(-5.0, -3.5))
    ctx = _ctx()
    model = to_gpu_model(P)
    gpu_render(ctx, model, cam, pose)
    assert _longest(ctx, cam) <= 512
    _no_sync(ctx, P["means"].shape[0], cam.width * cam.height, 4_000_000)
    big = dict(P)
    big["log_scales"] = (np.asarray(P["log_scales"]) + 0.8).astype(np.float32)
    model.flat.copy_(to_gpu_model(big).flat)
    got = gpu_render(ctx, model, cam, pose)
    from paper_2408_12677_gb300 import abi
    abi.gs_sync_status(ctx.handle)
    longest = _longest(ctx, cam)
    assert 512 < longest <= 1024, longest
    check_visit_order(ctx, -(-cam.width // 16) * -(-cam.height // 16))
    ref_ctx = _ctx()
    ref = gpu_render(ref_ctx, to_gpu_model(big), cam, pose)  # sync mode: counting-scatter binning
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
    ctx.close()
    ref_ctx.close()


def test_bucket_overflow_reports_capacity_and_falls_back():
    from paper_2408_12677_gb300 import abi
    P, cam, pose = _scene(seed=6, n=20000, log_scale_range=(-5.0, -3.5))
    ctx = _ctx()
    model = to_gpu_model(P)
    gpu_render(ctx, model, cam, pose)
    assert _longest(ctx, cam) <= 512
    _no_sync(ctx, P["means"].shape[0], cam.width * cam.height, 8_000_000)
    big = dict(P)
    big["log_scales"] = (np.asarray(P["log_scales"]) + 1.5).astype(np.float32)  # lists of 1025-4096
    model.flat.copy_(to_gpu_model(big).flat)
    gpu_render(ctx, model, cam, pose)
    with pytest.raises(abi.GsError) as ei:
        abi.gs_sync_status(ctx.handle)
    assert ei.value.status == abi.GS_ERR_CAPACITY and "bucket" in str(ei.value)
    # the context now bins by counting and scatter again, in no-sync mode too
    got = gpu_render(ctx, model, cam, pose)
    abi.gs_sync_status(ctx.handle)
    assert 1024 < _longest(ctx, cam) <= 4096
    ref_ctx = _ctx()
    ref = gpu_render(ref_ctx, to_gpu_model(big), cam, pose)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
    ctx.close()
    ref_ctx.close()


def test_bucket_binning_of_a_batch_of_views():
    w = workloads.tiny_multi_view(n=3000)
    ctx = _ctx()
    model = to_gpu_model(w.params)
    ref = _batched_render(ctx, model, w.views)
    npx = sum(v.cam.width * v.cam.height for v in w.views)
    _no_sync(ctx, w.n * len(w.views), npx, 1_000_000)
    got = _batched_render(ctx, model, w.views)
    check_visit_order(ctx, sum(-(-v.cam.width // 16) * -(-v.cam.height // 16) for v in w.views))
    for (a0, a1, a2), (b0, b1, b2) in zip(got, ref):
        np.testing.assert_array_equal(a0, b0)
        np.testing.assert_array_equal(a1, b1)
        np.testing.assert_array_equal(a2, b2)
    from paper_2408_12677_gb300 import abi
    abi.gs_sync_status(ctx.handle)
    ctx.close()


def test_bucket_size_follows_the_longest_list_any_sync_pass_saw():
    """A context that renders a map with long lists and then one with short
    lists in sync mode sizes its buckets from the long ones (or bins by
    counting): the no-sync pass of the first map overflows nothing and
    renders its sync-mode images."""
    from paper_2408_12677_gb300 import abi
    P, cam, pose = _scene(seed=6, n=20000, log_scale_range=(-5.0, -3.5))
    big = dict(P)
    big["log_scales"] = (np.asarray(P["log_scales"]) + 1.5).astype(np.float32)  # lists of 1025-4096
    ctx = _ctx()
    small_model, big_model = to_gpu_model(P), to_gpu_model(big)
    ref = gpu_render(ctx, big_model, cam, pose)
    assert _longest(ctx, cam) > 1024
    gpu_render(ctx, small_model, cam, pose)
    assert _longest(ctx, cam) <= 512
    _no_sync(ctx, P["means"].shape[0], cam.width * cam.height, 8_000_000)
    got = gpu_render(ctx, big_model, cam, pose)
    abi.gs_sync_status(ctx.handle)  # no bucket overflow
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
    ctx.close()


@pytest.mark.parametrize("which", ["single_view", "multi_view"])
def test_bucket_binning_at_full_size(which):
    """The bench's workloads (1200x680 with ~300k Gaussians; 8 views of
    640x480 to 1752x1168, 7.97M pixels, 500k Gaussians): a no-sync pass
    (bucket binning when every list of the sync pass is at most 2048 long)
    renders every pixel as the sync-mode pass does, bit for bit, and its
    visit order is a permutation of the tiles, longest class first."""
    import os
    from paper_2408_12677_gb300 import abi
    if which == "single_view":
        w = workloads.single_view()
    else:
        w = workloads.multi_view(workers=min(8, os.cpu_count() or 1))
    ctx = _ctx()
    model = to_gpu_model(w.params)
    T = sum(-(-v.cam.width // 16) * -(-v.cam.height // 16) for v in w.views)
    b0 = ctx.stats()["kernel_launches"]
    ref = _batched_render(ctx, model, w.views)
    n_sync = ctx.stats()["kernel_launches"] - b0
    longest = _longest_of(ctx, T)
    _no_sync(ctx, w.n * len(w.views), sum(v.cam.width * v.cam.height for v in w.views),
             int(abi.gs_get_stats(ctx.handle)["n_pairs"] * 1.5) + 4096)
    b1 = ctx.stats()["kernel_launches"]
    got = _batched_render(ctx, model, w.views)
    n_no_sync = ctx.stats()["kernel_launches"] - b1
    abi.gs_sync_status(ctx.handle)
    check_visit_order(ctx, T)
    if longest <= 2048:  # bucket binning engaged: no count, scan or scatter launch
        assert n_no_sync < n_sync
    for (a0, a1, a2), (b0, b1, b2) in zip(got, ref):
        np.testing.assert_array_equal(a0, b0)
        np.testing.assert_array_equal(a1, b1)
        np.testing.assert_array_equal(a2, b2)
    ctx.close()


def _longest_of(ctx, n_tiles):
    from paper_2408_12677_gb300 import abi
    r = torch.empty((n_tiles, 2), dtype=torch.int32, device="cuda")
    abi.gs_get_tile_ranges(ctx.handle, r)
    torch.cuda.synchronize()
    r = r.cpu().numpy().view(np.uint32).astype(np.int64)
    return int((r[:, 1] - r[:, 0]).max())
