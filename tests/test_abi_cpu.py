"""The C-ABI library builds, loads and exports every entry point that
include/gsplat.h declares; host-side argument handling needs no GPU."""
import ctypes as C
import os
import re

import pytest

from tests._util import ROOT, ensure_built

HEADER = os.path.join(ROOT, "include", "gsplat.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("gs_render_fwd", "gs_render_bwd", "gs_adam_step", "gs_loss_l1", "gs_bin_tiles",
                     "gs_ctx_create", "gs_ctx_destroy", "gs_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ensure_built()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2408_12677_gb300 import abi
    assert set(abi.EXPORTS) <= set(_declared())
    assert set(_declared()) <= set(abi.EXPORTS), "binding lacks a declared entry point"


def test_checked_build_exports_the_same_boundary():
    """libgsplat_checked.so (GS_CHECKED) declares itself and exports every
    entry point too; the normal library says it is not the checked one."""
    ensure_built()
    from paper_2408_12677_gb300 import abi
    checked = C.CDLL(abi.CHECKED_LIB_PATH)
    missing = [n for n in _declared() if not hasattr(checked, n)]
    assert not missing, missing
    checked.gs_bounds_checked.restype = C.c_int
    assert checked.gs_bounds_checked() == 1
    assert abi.gs_bounds_checked() is False


def test_struct_layouts_match_header_sizes():
    from paper_2408_12677_gb300 import abi
    assert C.sizeof(abi.gs_camera) == 24
    assert C.sizeof(abi.gs_viewmat) == 48
    assert C.sizeof(abi.gs_gaussians) == 5 * 8 + 8 + 8
    assert C.sizeof(abi.gs_raster_cfg) == 4 * 3 + 12 + 4 * 5
    assert C.sizeof(abi.gs_adam_cfg) == 40


def test_defaults_and_null_handling():
    lib = ensure_built()
    from paper_2408_12677_gb300 import abi
    c = abi.raster_cfg()
    assert (c.tile_w, c.tile_h, c.batch) == (16, 16, 32)
    assert abs(c.alpha_min - 1 / 255) < 1e-9 and abs(c.alpha_max - 0.99) < 1e-7
    assert abs(c.t_eps - 1e-4) < 1e-10 and abs(c.dilation - 0.3) < 1e-7 and abs(c.near_z - 0.2) < 1e-7
    a = abi.adam_cfg()
    assert (a.beta1, round(a.beta2, 6), a.zero_grads) == (pytest.approx(0.9), 0.999, 0)
    # a NULL context is rejected before any CUDA call
    for name in ("gs_ctx_destroy",):
        assert getattr(lib, name)(None) == 1
    cam = abi.make_camera(60, 60, 32, 24, 64, 48)
    assert lib.gs_loss_l1(None, C.byref(cam), None, None, None, None, 0.8, 0.2, None, None, None, None) == 1
    assert lib.gs_adam_step(None, None, None, None, None, 0, 0, C.byref(a), 1, None) == 1
    assert lib.gs_raster_cfg_default(None) == 1
    assert lib.gs_last_error(None) == b"null context"


def test_context_creation_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = ensure_built()
    h = C.c_void_p()
    st = lib.gs_ctx_create(C.byref(h), 0, 0)
    assert st in (2, 7) and h.value is None


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2408_12677_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_struct_layouts_match_the_compiled_header(tmp_path):
    """Every struct the binding passes by pointer has the size and field
    offsets a C compiler gives the header's declaration."""
    import shutil
    import subprocess
    from paper_2408_12677_gb300 import abi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [abi.gs_camera, abi.gs_viewmat, abi.gs_gaussians, abi.gs_grads, abi.gs_raster_cfg, abi.gs_adam_cfg,
               abi.gs_stats, abi.gs_tsdf_grid, abi.gs_alu_peaks]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gsplat.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, key, value = line.split()
        got[(name, key)] = int(value)
    for st in structs:
        name = st.__name__
        assert got[(name, "size")] == C.sizeof(st), name
        for field, _ in st._fields_:
            assert got[(name, field)] == getattr(st, field).offset, (name, field)
