"""Build libgsplat.so (the CUDA path and its C ABI) in-tree for sm_103a, and
its bounds-checked twin libgsplat_checked.so (compiled with GS_CHECKED:
every index read from memory is checked, see gs_bounds_checked).

Each translation unit under csrc/ is compiled by nvcc in parallel (both
variants in one pool) into _build/ and _build_checked/, then linked.  The
CUDA runtime is linked statically, so the libraries only need the driver.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgsplat.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libgsplat_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
# (library, object folder, extra flags) of each variant
VARIANTS = [(LIB, BUILD, []), (LIB_CHECKED, BUILD_CHECKED, ["-DGS_CHECKED"])]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgsplat")
    return path


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _compile(src: str, out_dir: str, extra) -> str:
    obj = os.path.join(out_dir, os.path.basename(src) + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if r.stderr.strip():
        sys.stderr.write(r.stderr)
    return obj


def _link(lib: str, objs) -> None:
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)


def build(verbose: bool = False, extra=(), checked: bool = True) -> str:
    """Compile every csrc/*.cu and link libgsplat.so (and, with `checked`,
    libgsplat_checked.so); returns the normal library's path."""
    variants = VARIANTS if checked else VARIANTS[:1]
    srcs = sources()
    jobs = []
    for _, out_dir, flags in variants:
        os.makedirs(out_dir, exist_ok=True)
        jobs += [(src, out_dir, [*flags, *extra]) for src in srcs]
    workers = max(1, min(len(jobs), os.cpu_count() or 8))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(lambda j: _compile(*j), jobs))
    for k, (lib, _, _) in enumerate(variants):
        _link(lib, objs[k * len(srcs):(k + 1) * len(srcs)])
        if verbose:
            print("built", lib)
    return LIB


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
