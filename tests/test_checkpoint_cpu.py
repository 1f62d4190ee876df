"""Checkpoint file format (host side): round trip, header checks, and the
rejection of foreign, newer or truncated files."""
import numpy as np
import pytest

from paper_2408_12677_gb300 import checkpoint as C


def _arrays(n, deg, seed=0):
    rng = np.random.default_rng(seed)
    size = n * C.floats_per_gaussian(deg)
    return [rng.standard_normal(size).astype(np.float32) for _ in range(3)]


@pytest.mark.parametrize("n,deg,live,step", [(1, 0, 1, 0), (37, 3, 20, 12345), (5, 1, 0, 7)])
def test_round_trip(tmp_path, n, deg, live, step):
    flat, m, v = _arrays(n, deg, n)
    p = str(tmp_path / "map.ckpt")
    C.save_map(p, flat, m, v, n, deg, step, live)
    d = C.load_map(p)
    assert (d["n_slots"], d["n_live"], d["sh_degree"], d["step"]) == (n, live, deg, step)
    for key, a in (("flat", flat), ("m", m), ("v", v)):
        assert np.array_equal(d[key], a)
    import os
    assert os.path.getsize(p) == C.HEADER_BYTES + 3 * 4 * n * C.floats_per_gaussian(deg)


def test_rejects_bad_files(tmp_path):
    flat, m, v = _arrays(4, 2)
    p = str(tmp_path / "map.ckpt")
    C.save_map(p, flat, m, v, 4, 2, 3)
    raw = open(p, "rb").read()
    for name, data, msg in [("short", raw[:40], "header"), ("trunc", raw[:-4], "size"),
                            ("long", raw + b"\0", "size"), ("magic", b"X" + raw[1:], "not a"),
                            ("version", raw[:8] + (99).to_bytes(4, "little") + raw[12:], "version")]:
        q = str(tmp_path / name)
        open(q, "wb").write(data)
        with pytest.raises(ValueError, match=msg):
            C.load_map(q)
    with pytest.raises(ValueError):
        C.save_map(p, flat, m, v, 4, 2, 3, n_live=5)
    with pytest.raises(ValueError):
        C.save_map(p, flat[:-1], m, v, 4, 2, 3)
