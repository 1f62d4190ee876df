"""Checkpoint / resume of a trainer and of the streaming loop, the
non-finite check and the injected allocation failure (the context must stay
usable)."""
import numpy as np
import pytest
import torch

from synth import workloads
from tests._util import ensure_built, gpu_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return ensure_built()


def _trainer(w, ctx=None):
    from paper_2408_12677_gb300.torch_api import Context, GaussianModel, Trainer
    v = w.views[0]
    return Trainer(GaussianModel(w.params), v.cam, v.pose.R, v.pose.t, ctx=ctx or Context(0))


def _targets(w):
    v = w.views[0]
    return torch.as_tensor(v.target_rgb, device="cuda"), torch.as_tensor(v.target_depth, device="cuda")


def test_trainer_checkpoint_round_trip(lib, tmp_path):
    w = workloads.tiny_random(seed=41, n=600, sh_degree=1, sh_rest_std=0.05)
    trgb, tdep = _targets(w)
    a = _trainer(w)
    for _ in range(3):
        a.step(trgb, tdep)
    path = str(tmp_path / "map.ckpt")
    a.save(path)
    b = _trainer(w)
    b.load(path)
    for x, y in ((a.model.flat, b.model.flat), (a.model.m, b.model.m), (a.model.v, b.model.v)):
        assert torch.equal(x, y)
    assert a.step_count == b.step_count == 3
    la, lb = float(a.step(trgb, tdep)), float(b.step(trgb, tdep))
    assert la == lb  # same parameters: the forward pass and its fixed-order loss are identical
    # a map of another size is refused
    c = _trainer(workloads.tiny_random(seed=41, n=300, sh_degree=1))
    with pytest.raises(ValueError):
        c.load(path)


def test_streaming_resume(lib, tmp_path):
    from paper_2408_12677_gb300.streaming import StreamingOptimizer, load_stream, save_stream
    st = workloads.streaming(n_frames=40, width=96, height=64, f=60.0)
    sp = dict(var_thr=0.02, max_size=32, min_size=2)

    def make():
        return StreamingOptimizer(st.cam, 1, None, iters=2, n_past=2, capacity=256, rng_seed=9, seeding=sp)

    frames = [0, 3, 6, 9, 12, 15]
    a = make()
    for k in frames[:4]:
        a.process_frame(*st.frame(k), st.poses[k])
    path = str(tmp_path / "stream.ckpt")
    save_stream(a, path)
    ref = [a.process_frame(*st.frame(k), st.poses[k]) for k in frames[4:]]
    b = make()
    load_stream(b, path, lambda i: (*st.frame(frames[i]), st.poses[frames[i]]))
    assert b.map.n == 0 or b.keyframe_ids == a.keyframe_ids[:len(b.keyframe_ids)]
    got = [b.process_frame(*st.frame(k), st.poses[k]) for k in frames[4:]]
    for r, g in zip(ref, got):
        assert (g.new_gaussians, g.n_gaussians, g.tsdf_blocks, g.tsdf_touched, g.views_per_iter) == \
            (r.new_gaussians, r.n_gaussians, r.tsdf_blocks, r.tsdf_touched, r.views_per_iter)
        assert g.loss == pytest.approx(r.loss, rel=1e-3)
    assert b.keyframe_ids == a.keyframe_ids
    # a crash between the two renames of a later save leaves the new map file
    # beside the old state file: the pair is refused
    import shutil
    old_state = str(tmp_path / "old.state.npz")
    shutil.copy(path + ".state.npz", old_state)
    save_stream(a, path)
    shutil.copy(old_state, path + ".state.npz")
    with pytest.raises(ValueError, match="different checkpoints"):
        load_stream(make(), path, lambda i: (*st.frame(frames[i]), st.poses[frames[i]]))


def test_nonfinite_count(lib):
    from paper_2408_12677_gb300 import abi
    from paper_2408_12677_gb300.torch_api import Context
    ctx = Context(0)
    x = torch.randn(1_000_003, device="cuda")
    assert abi.gs_count_nonfinite(ctx.handle, x) == 0
    x[[5, 77, 1_000_002]] = float("nan")
    x[123] = float("inf")
    x[124] = -float("inf")
    assert abi.gs_count_nonfinite(ctx.handle, x) == 5
    assert abi.gs_count_nonfinite(ctx.handle, x[:0]) == 0
    w = workloads.tiny_random(seed=3, n=200)
    tr = _trainer(w, ctx)
    tr.step(*_targets(w))
    assert tr.nonfinite() == 0
    tr.model.p["means"][7, 1] = float("nan")
    assert tr.nonfinite() == 1


def test_injected_alloc_failure_leaves_context_usable(lib):
    from paper_2408_12677_gb300 import abi
    from paper_2408_12677_gb300.torch_api import Context, GaussianModel
    small = workloads.tiny_random(seed=5, n=100)
    big = workloads.tiny_random(seed=6, n=20_000)
    ctx = Context(0)
    gpu_render(ctx, GaussianModel(small.params), small.views[0].cam, small.views[0].pose)
    abi.gs_ctx_inject_alloc_failure(ctx.handle, 1)
    m_big = GaussianModel(big.params)
    with pytest.raises(abi.GsError) as err:
        gpu_render(ctx, m_big, big.views[0].cam, big.views[0].pose)
    assert "injected" in str(err.value)
    got = gpu_render(ctx, m_big, big.views[0].cam, big.views[0].pose)
    want = gpu_render(Context(0), m_big, big.views[0].cam, big.views[0].pose)
    for g, r in zip(got, want):
        assert np.array_equal(g, r)
