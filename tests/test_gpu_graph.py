"""One training iteration captured as a CUDA graph (no-sync mode, reserved
pair buffers, device-side Adam step counter) gives the same parameters and
moments as the same number of eager iterations."""
import numpy as np
import pytest
import torch

from synth import workloads
from tests._util import compare, ensure_built

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,deg", [(1000, 0), (7, 3)])
def test_graph_replay_matches_eager(seed, deg):
    ensure_built()
    from paper_2408_12677_gb300.torch_api import Context, GaussianModel, Trainer
    w = workloads.tiny_random(seed=seed, sh_degree=deg, sh_rest_std=0.1 if deg else 0.0)
    v = w.views[0]
    trgb = torch.as_tensor(v.target_rgb, device="cuda")
    tdep = torch.as_tensor(v.target_depth, device="cuda")
    A, B = GaussianModel(w.params), GaussianModel(w.params)
    ta = Trainer(A, v.cam, v.pose.R, v.pose.t, ctx=Context(0))
    tb = Trainer(B, v.cam, v.pose.R, v.pose.t, ctx=Context(0))
    for _ in range(4):
        ta.step(trgb, tdep)
    tb.step(trgb, tdep)
    tb.capture(trgb, tdep)  # one eager no-sync iteration, then capture
    tb.replay()
    tb.replay()
    torch.cuda.synchronize()
    tb.check_capacity()
    assert ta.step_count == tb.step_count == 4
    for name, x, y in (("p", A.flat, B.flat), ("m", A.m, B.m), ("v", A.v, B.v)):
        xa = x.cpu().numpy()
        compare(name, y.cpu().numpy(), xa, 1e-4, 1e-6 * np.abs(xa).max() + 1e-12, 1e-5)
    assert abs(float(ta.loss) - float(tb.loss)) <= 1e-5 * abs(float(ta.loss))
