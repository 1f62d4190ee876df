"""Checkpoint and resume of a Gaussian map with its Adam state.

One flat little-endian binary file: a 64-byte header (magic, format version,
SH degree, slots N, live Gaussians, Adam step) followed by the parameters,
the first and the second Adam moment, each N (11 + 3K) float32 in the flat
layout of the C ABI (means | log-scales | quaternions | opacity logits |
SH).  The file is written to a temporary name and renamed, so a reader never
sees a partial checkpoint.
"""
from __future__ import annotations

import os
import struct

import numpy as np

MAGIC = b"GSFCKPT\0"
VERSION = 1
_HEADER = struct.Struct("<8sIIQQQ24x")  # 64 bytes
HEADER_BYTES = _HEADER.size


def floats_per_gaussian(sh_degree: int) -> int:
    return 11 + 3 * (sh_degree + 1) ** 2


def _host(a) -> np.ndarray:
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, np.float32).ravel()


def save_map(path: str, flat, m, v, n_slots: int, sh_degree: int, step: int, n_live: int | None = None) -> None:
    """Writes the map (flat parameters, Adam moments m and v) of n_slots
    Gaussians, n_live of them in use (default all), at Adam step ``step``."""
    n_live = n_slots if n_live is None else int(n_live)
    size = int(n_slots) * floats_per_gaussian(sh_degree)
    arrays = [_host(a) for a in (flat, m, v)]
    for a in arrays:
        if a.size != size:
            raise ValueError(f"expected {size} floats per array, got {a.size}")
    if not 0 <= n_live <= n_slots or step < 0 or not 0 <= sh_degree <= 3:
        raise ValueError("bad checkpoint header values")
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        f.write(_HEADER.pack(MAGIC, VERSION, int(sh_degree), int(n_slots), n_live, int(step)))
        for a in arrays:
            a.tofile(f)
    os.replace(tmp, path)


def load_map(path: str) -> dict:
    """Reads a checkpoint: {flat, m, v (float32 host arrays), n_slots,
    n_live, sh_degree, step}.  Raises ValueError on a foreign, newer or
    truncated file."""
    with open(path, "rb") as f:
        head = f.read(HEADER_BYTES)
        if len(head) != HEADER_BYTES:
            raise ValueError("checkpoint too short for its header")
        magic, version, deg, n_slots, n_live, step = _HEADER.unpack(head)
        if magic != MAGIC:
            raise ValueError("not a Gaussian map checkpoint")
        if version != VERSION:
            raise ValueError(f"checkpoint format version {version}, this reader knows {VERSION}")
        if deg > 3 or n_live > n_slots:
            raise ValueError("corrupt checkpoint header")
        size = n_slots * floats_per_gaussian(deg)
        data = np.fromfile(f, np.float32, 3 * size)
        if data.size != 3 * size or f.read(1):
            raise ValueError("checkpoint size does not match its header")
    return {"flat": data[:size], "m": data[size:2 * size], "v": data[2 * size:], "n_slots": int(n_slots),
            "n_live": int(n_live), "sh_degree": int(deg), "step": int(step)}
