"""TSDF map (Sec. III-B.1) in device memory, fused frame by frame through
the C ABI (gs_tsdf_integrate), with the voxel-weight novelty check of the
seeding (gs_seed_tsdf, Sec. III-B.2).

The host side only sizes buffers: before a frame the hash table is grown
(rehashed on the device) until no insert of that frame can fail, and when a
frame hands out more block slots than the pool holds the pool is grown and
the integration re-run for the new slots only.  Every step of the fusion
runs in the CUDA kernels.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import abi

FUSION = {"printed": 0, "unit": 1}


def _pow2(n: int) -> int:
    return 1 << max(1, int(n - 1).bit_length())


def band_samples(truncation: float, voxel_size: float) -> int:
    """Samples per ray of the allocation (as gs_tsdf_integrate takes them):
    n + 1 with n = ceil(eps / 2s), float32 eps and s."""
    e, s = float(np.float32(truncation)), float(np.float32(voxel_size))
    return max(1, math.ceil(e / (2.0 * s) - 1e-6)) + 1


class TSDFGrid:
    """Single-resolution TSDF grid: voxels of ``voxel_size`` metres in blocks
    of 8^3, truncation ``truncation`` metres, weights capped at
    ``max_weight`` (Eq. 8), Eq. 9 as printed (``fusion="printed"``) or with a
    unit measurement weight (``"unit"``)."""

    def __init__(self, ctx, voxel_size: float = 0.01, truncation: float = 0.08, max_weight: float = 100.0,
                 fusion: str = "printed", capacity: int = 1 << 14, table_size: int = 1 << 16, device=None):
        self.ctx = ctx
        self.device = torch.device(device or "cuda")
        self.voxel_size = float(np.float32(voxel_size))
        self.truncation = float(np.float32(truncation))
        self.max_weight = float(max_weight)
        self.fusion = FUSION[fusion]
        self.frame = 0
        self.n_blocks = 0
        self.updated = 0
        self.counters = torch.zeros(4, dtype=torch.int32, device=self.device)
        self._new_table(_pow2(table_size))
        self._new_pool(int(capacity))
        self.last = {}

    # -- buffers -----------------------------------------------------------
    def _new_table(self, size: int):
        self.table_size = size
        self.keys = torch.full((size,), -1, dtype=torch.int64, device=self.device)
        self.slots = torch.empty(size, dtype=torch.int32, device=self.device)
        self.stamps = torch.zeros(size, dtype=torch.int32, device=self.device)
        self.touched = torch.empty(size // 2, dtype=torch.int32, device=self.device)

    def _new_pool(self, capacity: int):
        self.capacity = capacity
        self.voxels = torch.zeros((capacity, 512, 2), dtype=torch.float32, device=self.device)
        self.claims = torch.full((capacity, 512), -1, dtype=torch.int32, device=self.device)

    def struct(self) -> abi.gs_tsdf_grid:
        return abi.gs_tsdf_grid(self.keys.data_ptr(), self.slots.data_ptr(), self.stamps.data_ptr(),
                                self.voxels.data_ptr(), self.claims.data_ptr(), self.touched.data_ptr(),
                                self.counters.data_ptr(), self.table_size, self.capacity, self.voxel_size,
                                self.truncation, self.max_weight, self.fusion)

    @property
    def band_samples(self) -> int:
        return band_samples(self.truncation, self.voxel_size)

    def reserve(self, n_pixels: int):
        """Grow the hash table so that a frame of ``n_pixels`` cannot fill it
        (at most one new block per band sample)."""
        need = 2 * (self.n_blocks + n_pixels * self.band_samples)
        if need <= self.table_size:
            return
        old = self.struct()
        keep = (self.keys, self.slots, self.stamps, self.touched)
        self._new_table(_pow2(need))
        abi.gs_tsdf_rehash(self.ctx.handle, old, self.struct())
        torch.cuda.current_stream().synchronize()
        del keep

    def grow_pool(self, need: int):
        cap = _pow2(max(need + need // 4, 2 * self.capacity))
        vox, claims = self.voxels, self.claims
        self._new_pool(cap)
        self.voxels[:vox.shape[0]] = vox
        self.claims[:claims.shape[0]] = claims

    # -- fusion ------------------------------------------------------------
    def integrate(self, depth: torch.Tensor, cam: abi.gs_camera, view: abi.gs_viewmat) -> dict:
        """Fuse one depth image [H, W] (device float32) seen with the
        world-to-camera pose ``view``; returns the frame's counts and the
        CUDA-event time of its kernels (ms)."""
        self.reserve(int(cam.width) * int(cam.height))
        self.frame += 1
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record()
        abi.gs_tsdf_integrate(self.ctx.handle, self.struct(), depth, cam, view, self.frame, 0)
        ev[1].record()
        c, st = abi.gs_tsdf_counters(self.ctx.handle, self.struct())
        ms = ev[0].elapsed_time(ev[1])
        if c[2]:
            raise RuntimeError(f"TSDF table overflow ({c[2]} failed inserts)")
        if c[0] > self.capacity:
            old = self.capacity
            self.grow_pool(c[0])
            ev[2].record()
            abi.gs_tsdf_integrate(self.ctx.handle, self.struct(), depth, cam, view, self.frame, old)
            ev[3].record()
            c, st = abi.gs_tsdf_counters(self.ctx.handle, self.struct())
            if st != abi.GS_OK:
                raise RuntimeError("TSDF integration failed after growing the pool")
            ms += ev[2].elapsed_time(ev[3])
        new_blocks = c[0] - self.n_blocks
        self.n_blocks = c[0]
        self.last = {"blocks": c[0], "new_blocks": new_blocks, "touched": c[1], "updated": c[3] - self.updated,
                     "ms": ms}
        self.updated = c[3]
        return self.last

    def query(self, points: torch.Tensor):
        """(tsdf, weight) of the voxels holding world points [n, 3]."""
        n = points.shape[0]
        ts = torch.empty(n, dtype=torch.float32, device=self.device)
        ws = torch.empty(n, dtype=torch.float32, device=self.device)
        abi.gs_tsdf_query(self.ctx.handle, self.struct(), points.contiguous(), ts, ws)
        return ts, ws

    def seed(self, rgb, depth, cam, view, sh_degree, var_thr, max_size, min_size, means, log_scales, quats,
             opacity_logits, sh, capacity) -> int:
        """Quadtree seeding gated by the voxel weights (weight 1 = first seen
        by this frame's integration); see abi.gs_seed_tsdf."""
        return abi.gs_seed_tsdf(self.ctx.handle, rgb, depth, self.struct(), cam, view, sh_degree, var_thr, max_size,
                                min_size, means, log_scales, quats, opacity_logits, sh, capacity)

    # -- checkpoint --------------------------------------------------------
    def state(self) -> dict:
        """Host copy of the grid for a checkpoint: the live (key, slot) pairs,
        the voxels of the allocated slots, the frame counter and counters."""
        torch.cuda.synchronize()
        keys = self.keys.cpu().numpy()
        live = np.nonzero(keys != -1)[0]
        return {"keys": keys[live], "slots": self.slots.cpu().numpy()[live],
                "voxels": self.voxels[:self.n_blocks].cpu().numpy(), "frame": self.frame,
                "n_blocks": self.n_blocks, "updated": self.updated,
                "params": [self.voxel_size, self.truncation, self.max_weight, self.fusion]}

    def load_state(self, st: dict) -> None:
        """Restores ``state()``: a table sized for the blocks, rebuilt on the
        device from the saved (key, slot) pairs (gs_tsdf_rehash from a
        compact table), and the voxels."""
        n_blocks = int(st["n_blocks"])
        self.voxel_size, self.truncation, self.max_weight, self.fusion = (float(st["params"][0]),
                                                                          float(st["params"][1]),
                                                                          float(st["params"][2]),
                                                                          int(st["params"][3]))
        self._new_pool(max(_pow2(max(n_blocks, 1)), self.capacity))
        if n_blocks:
            self.voxels[:n_blocks] = torch.as_tensor(np.asarray(st["voxels"], np.float32), device=self.device)
        self.n_blocks, self.updated, self.frame = n_blocks, int(st["updated"]), int(st["frame"])
        self._new_table(_pow2(max(2 * n_blocks, 1 << 16)))
        keys = np.asarray(st["keys"], np.int64)
        if keys.size:
            size = _pow2(max(keys.size, 2))
            src_keys = torch.full((size,), -1, dtype=torch.int64, device=self.device)
            src_slots = torch.zeros(size, dtype=torch.int32, device=self.device)
            src_keys[:keys.size] = torch.as_tensor(keys, device=self.device)
            src_slots[:keys.size] = torch.as_tensor(np.asarray(st["slots"], np.int32), device=self.device)
            src = self.struct()
            src.keys, src.slots, src.table_size = src_keys.data_ptr(), src_slots.data_ptr(), size
            abi.gs_tsdf_rehash(self.ctx.handle, src, self.struct())
            torch.cuda.synchronize()
        c = torch.tensor([n_blocks, 0, 0, self.updated], dtype=torch.int64).to(torch.int32)
        self.counters.copy_(c.to(self.device))

    # -- read-out ----------------------------------------------------------
    def blocks(self) -> dict:
        """{(bx, by, bz): (tsdf [8, 8, 8], weight [8, 8, 8])} indexed [z, y, x]
        (host copy, for checks and export)."""
        keys = self.keys.cpu().numpy().view(np.uint64)
        live = np.nonzero(keys != np.uint64(0xFFFFFFFFFFFFFFFF))[0]
        slots = self.slots.cpu().numpy()[live]
        vox = self.voxels.cpu().numpy()
        out = {}
        bias = 1 << 20
        for k, sl in zip(keys[live].tolist(), slots.tolist()):
            if sl >= self.capacity:
                continue
            b = (((k >> 42) & 0x1FFFFF) - bias, ((k >> 21) & 0x1FFFFF) - bias, (k & 0x1FFFFF) - bias)
            v = vox[sl].reshape(8, 8, 8, 2)
            out[b] = (v[..., 0], v[..., 1])
        return out
