"""The bounds-checked build (libgsplat_checked.so, GS_CHECKED) on the GPU:
the same calls as the normal build (tests/_checked_run.py: a small map with
loss, backward and two training steps, a ragged image, a batched pair of
views, the radix binning) meet no out-of-bounds index, give the same
forward images bit for bit and the same gradients up to float32 atomics
order, and a bounds fault set from the host is reported once as
GS_ERR_BOUNDS.  Each build runs in its own process."""
import os
import subprocess
import sys

import numpy as np
import pytest

from tests._util import ROOT, ensure_built

pytestmark = pytest.mark.gpu


def _run(which, path):
    r = subprocess.run([sys.executable, "-m", "tests._checked_run", which, str(path)], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return dict(np.load(path))


def test_checked_build_matches_and_reports(tmp_path):
    ensure_built()
    normal = _run("normal", tmp_path / "normal.npz")
    checked = _run("checked", tmp_path / "checked.npz")
    assert not bool(normal["checked"]) and bool(checked["checked"])
    for out in (normal, checked):
        assert bool(out["bounds_clean"])
        assert bool(out["injected_reported"])
    for key in sorted(normal):
        if key.endswith(("_color", "_depth", "_alpha")) or key.startswith("batched_color"):
            np.testing.assert_array_equal(checked[key], normal[key], err_msg=key)
    np.testing.assert_allclose(checked["small_loss"], normal["small_loss"], rtol=1e-6)
    for key in ("small_grad", "batched_grad"):
        a, b = checked[key], normal[key]
        err = np.abs(a - b)
        assert (err <= 1e-4 * np.abs(b) + 1e-6 * np.abs(b).max()).all(), (key, float(err.max()))
    a, b = checked["small_params"], normal["small_params"]
    bad = np.abs(a - b) > 1e-5 * np.abs(b) + 1e-6 * np.abs(b).max()
    assert bad.sum() <= max(2, int(1e-4 * a.size)), int(bad.sum())
