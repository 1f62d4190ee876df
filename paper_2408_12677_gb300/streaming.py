"""Per-frame streaming optimisation: GSFusion's online loop around the hot
path (Sec. III-B).  For every incoming RGB-D frame:

1. fuse the depth image into the TSDF grid (gs_tsdf_integrate, Eq. 6-9);
2. seed new Gaussians at the quadtree leaves whose back-projected centre
   falls in a voxel first seen by this frame (weight 1, at most one Gaussian
   per voxel: gs_seed_tsdf, Sec. III-B.2).  ``novelty="alpha"`` instead
   renders the current map at the frame's pose and seeds where its alpha is
   below 0.5 (gs_seed_quadtree), and a host ``seed_fn`` seeds with that mask
   on the CPU;
3. append them to the map (capacity-doubling buffers, Adam moments of the
   new Gaussians zero);
4. keep the frame as a keyframe when it added more than 50 Gaussians
   (Sec. IV-A.4);
5. run ``iters`` optimisation iterations, each one batched over the current
   frame and up to ``n_past`` random earlier keyframes (Sec. III-B.3 revisits
   keyframes; one Adam step per iteration on the summed loss).

The map lives in flat buffers of a fixed capacity: slots [0, n) hold the
Gaussians, the others are inert (opacity logit and log-scales -30, so the
projection gives them no tile and their gradient, hence their Adam update,
is zero).  The kernels always run over the whole capacity, which only changes
when the map doubles.  All per-Gaussian and per-voxel arithmetic runs in
libgsplat; this module moves buffers and chooses views.
"""
from __future__ import annotations

import dataclasses
import os
import time

import numpy as np
import torch

from . import abi
from .torch_api import PARAM_NAMES, Context, GaussianModel, camera_struct, flat_sizes, n_sh
from .tsdf import TSDFGrid

INERT_LOGIT = -30.0
INERT_LOG_SCALE = -30.0
NOVELTY_ALPHA = 0.5
KEYFRAME_MIN_NEW = 50


def inert_params(n: int, sh_degree: int) -> dict:
    """Host parameters of n inert slots."""
    K = n_sh(sh_degree)
    quats = np.zeros((n, 4), np.float32)
    quats[:, 0] = 1.0
    return {"means": np.zeros((n, 3), np.float32),
            "log_scales": np.full((n, 3), INERT_LOG_SCALE, np.float32), "quats": quats,
            "opacity_logits": np.full(n, INERT_LOGIT, np.float32), "sh": np.zeros((n, K, 3), np.float32),
            "sh_degree": sh_degree}


def novelty_mask(alpha: np.ndarray, thr: float = NOVELTY_ALPHA) -> np.ndarray:
    """Pixels the map does not cover yet (rendered alpha below ``thr``)."""
    return np.asarray(alpha) < thr


def pick_views(rng: np.random.Generator, n_keyframes: int, current_is_keyframe: bool, n_past: int) -> list:
    """Indices of the earlier keyframes an iteration optimises besides the
    current frame: up to n_past distinct ones, drawn uniformly (the current
    frame, if it became a keyframe, is the last one and is not drawn)."""
    pool = n_keyframes - (1 if current_is_keyframe else 0)
    if pool <= 0 or n_past <= 0:
        return []
    return sorted(rng.choice(pool, size=min(n_past, pool), replace=False).tolist())


class GrowingMap:
    """Gaussian map in capacity-doubling flat buffers (parameters, gradient,
    Adam moments); ``n`` live slots, the rest inert."""

    def __init__(self, sh_degree: int, capacity: int = 1 << 16, device: int = 0):
        self.sh_degree = int(sh_degree)
        self.device = device
        self.n = 0
        self.model = GaussianModel(inert_params(int(capacity), self.sh_degree), device=f"cuda:{device}")

    @property
    def capacity(self) -> int:
        return self.model.n

    def _grow(self, need: int):
        cap = self.capacity
        while cap < need:
            cap *= 2
        old = self.model
        new = GaussianModel(inert_params(cap, self.sh_degree), device=f"cuda:{self.device}")
        for name in PARAM_NAMES:  # copy the first old.n slots of every block
            new.p[name][:old.n].copy_(old.p[name])
        for src, dst in ((old.m, new.m), (old.v, new.v)):
            so = do = 0
            for size_old, size_new in zip(flat_sizes(old.n, self.sh_degree), flat_sizes(cap, self.sh_degree)):
                dst[do:do + size_old].copy_(src[so:so + size_old])
                so += size_old
                do += size_new
        self.model = new

    def append(self, params: dict) -> int:
        """Write k new Gaussians into slots [n, n + k) (moments zero)."""
        k = int(np.asarray(params["means"]).shape[0])
        if k == 0:
            return 0
        if self.n + k > self.capacity:
            self._grow(self.n + k)
        m = self.model
        dev = m.flat.device
        a, b = self.n, self.n + k
        for name in PARAM_NAMES:
            m.p[name][a:b].copy_(torch.as_tensor(np.asarray(params[name], np.float32), device=dev))
        off = 0
        for size in flat_sizes(m.n, self.sh_degree):  # zero the new slots' moments in every block
            per = size // m.n
            m.m[off + a * per:off + b * per].zero_()
            m.v[off + a * per:off + b * per].zero_()
            off += size
        self.n = b
        return k

    def live_params(self) -> dict:
        """Host copy of the live Gaussians' parameters."""
        out = {k: v[:self.n].detach().cpu().numpy().copy() for k, v in self.model.p.items()}
        out["sh_degree"] = self.sh_degree
        return out


@dataclasses.dataclass
class Keyframe:
    cam: object
    view: abi.gs_viewmat
    rgb: torch.Tensor    # [3, H, W] device
    depth: torch.Tensor  # [H, W] device


@dataclasses.dataclass
class FrameStats:
    index: int
    new_gaussians: int
    n_gaussians: int
    capacity: int
    keyframe: bool
    views_per_iter: list
    loss: float
    gpu_ms: float        # CUDA-event time of the frame's optimisation iterations
    host_ms: float       # wall time of the whole frame (fusion, seeding, upload, iterations)
    tsdf_ms: float = 0.0  # CUDA-event time of the frame's TSDF fusion (allocation + integration)
    tsdf_blocks: int = 0  # allocated voxel blocks after the frame
    tsdf_touched: int = 0  # blocks the frame allocated or updated
    tsdf_updated: int = 0  # voxels the frame updated


class StreamingOptimizer:
    """The per-frame loop over one camera model (all frames share it)."""

    def __init__(self, cam, sh_degree: int, seed_fn=None, iters: int = 10, n_past: int = 4, capacity: int = 1 << 16,
                 raster_cfg=None, adam_cfg=None, w_color: float = 0.8, w_depth: float = 0.2, rng_seed: int = 0,
                 device: int = 0, ctx: Context | None = None, seeding=None, novelty: str = "tsdf", tsdf=None):
        """``seed_fn(rgb, depth, cam, pose, mask) -> params`` seeds on the host
        with the rendered-alpha mask; without it the frame is seeded on the
        device with ``seeding`` = dict(var_thr, max_size, min_size) and the
        ``novelty`` rule: "tsdf" (the voxel weights of the TSDF grid built
        from ``tsdf`` = dict(voxel_size, truncation, max_weight, fusion)) or
        "alpha" (rendered alpha < 0.5)."""
        if novelty not in ("tsdf", "alpha"):
            raise ValueError(f"novelty must be 'tsdf' or 'alpha', not {novelty!r}")
        self.cam = cam
        self.cam_s = camera_struct(cam)
        self.seed_fn = seed_fn
        self.novelty = "alpha" if seed_fn is not None else novelty
        self.seeding = {"var_thr": 0.01, "max_size": 64, "min_size": 1, **(seeding or {})}
        self.iters, self.n_past = int(iters), int(n_past)
        self.map = GrowingMap(sh_degree, capacity, device)
        self.ctx = ctx or Context(device)
        self.rcfg = raster_cfg or abi.raster_cfg()
        self.acfg = adam_cfg or abi.adam_cfg(zero_grads=1)
        self.w_color, self.w_depth = float(w_color), float(w_depth)
        self.rng = np.random.default_rng(rng_seed)
        self.keyframes: list[Keyframe] = []
        self.keyframe_ids: list[int] = []  # position of each keyframe in the processed sequence
        self.step = 0
        H, W = cam.height, cam.width
        dev = torch.device("cuda", device)
        slots = 1 + self.n_past
        self.color = [torch.empty((3, H, W), device=dev) for _ in range(slots)]
        self.depth = [torch.empty((H, W), device=dev) for _ in range(slots)]
        self.alpha = [torch.empty((H, W), device=dev) for _ in range(slots)]
        self.dLdc = [torch.empty((3, H, W), device=dev) for _ in range(slots)]
        self.dLdd = [torch.empty((H, W), device=dev) for _ in range(slots)]
        self.loss = torch.zeros(1, device=dev)
        self.frame_index = 0
        self.tsdf = None
        if self.novelty == "tsdf":
            self.tsdf = TSDFGrid(self.ctx, device=dev, **{"voxel_size": 0.01, "truncation": 0.08,
                                                          "max_weight": 100.0, **(tsdf or {})})

    def render_alpha(self, view) -> np.ndarray:
        """Alpha image of the current map at ``view`` (host array)."""
        if self.map.n == 0:
            return np.zeros((self.cam.height, self.cam.width), np.float32)
        abi.gs_render_fwd(self.ctx.handle, self.map.model.gaussians(), self.cam_s, view, self.rcfg, None, None,
                          self.alpha[0])
        return self.alpha[0].cpu().numpy()

    def iterate(self, views: list[Keyframe]):
        """One batched optimisation iteration over ``views`` (gs_train_step_batched)."""
        m = self.map.model
        V = len(views)
        self.step += 1
        abi.gs_train_step_batched(self.ctx.handle, m.gaussians(), [self.cam_s] * V, [k.view for k in views], self.rcfg,
                                  [k.rgb for k in views], [k.depth for k in views], self.w_color, self.w_depth,
                                  self.loss, m.flat, m.m, m.v, self.acfg, self.step)

    def seed_on_device(self, cur: "Keyframe") -> int:
        """Novelty seeding of the frame on the device (gs_seed_tsdf after the
        frame's TSDF fusion, or gs_seed_quadtree with the rendered alpha) into
        the map's free slots, growing the map when they do not suffice."""
        h = self.ctx.handle
        alpha = None
        if self.novelty == "alpha" and self.map.n > 0:
            abi.gs_render_fwd(h, self.map.model.gaussians(), self.cam_s, cur.view, self.rcfg, None, None,
                              self.alpha[0])
            alpha = self.alpha[0]
        sp = self.seeding
        for _ in range(2):
            m, n = self.map.model, self.map.n
            rows = (m.p["means"][n:], m.p["log_scales"][n:], m.p["quats"][n:], m.p["opacity_logits"][n:],
                    m.p["sh"][n:], m.n - n)
            if self.novelty == "tsdf":
                k = self.tsdf.seed(cur.rgb, cur.depth, self.cam_s, cur.view, self.map.sh_degree, sp["var_thr"],
                                   sp["max_size"], sp["min_size"], *rows)
            else:
                k = abi.gs_seed_quadtree(h, cur.rgb, cur.depth, alpha, NOVELTY_ALPHA, self.cam_s, cur.view,
                                         self.map.sh_degree, sp["var_thr"], sp["max_size"], sp["min_size"], *rows)
            if k >= 0:
                self.map.n += k
                return k
            self.map._grow(n - k - 1)  # -k - 1 = the number of new Gaussians
        raise RuntimeError("seeding did not fit after growing the map")

    def process_frame(self, rgb: np.ndarray, depth: np.ndarray, pose) -> FrameStats:
        """rgb [H, W, 3] in [0, 1], depth [H, W] (0 = invalid), pose: world-to-camera (R, t)."""
        t0 = time.perf_counter()
        view = abi.make_viewmat(pose.R, pose.t)
        dev = self.map.model.flat.device
        cur = Keyframe(self.cam, view, torch.as_tensor(np.ascontiguousarray(np.transpose(rgb, (2, 0, 1)), np.float32),
                                                        device=dev),
                       torch.as_tensor(np.ascontiguousarray(depth, np.float32), device=dev))
        fused = {}
        if self.tsdf is not None:
            fused = self.tsdf.integrate(cur.depth, self.cam_s, view)
        if self.seed_fn is None:
            k = self.seed_on_device(cur)
        else:
            alpha = self.render_alpha(view)
            k = self.map.append(self.seed_fn(rgb, depth, self.cam, pose, novelty_mask(alpha)))
        is_key = k > KEYFRAME_MIN_NEW or not self.keyframes
        if is_key:
            self.keyframes.append(cur)
            self.keyframe_ids.append(self.frame_index)
        sizes = []
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(self.iters):
            past = [self.keyframes[i] for i in pick_views(self.rng, len(self.keyframes), is_key, self.n_past)]
            views = [cur] + past
            sizes.append(len(views))
            self.iterate(views)
        ev1.record()
        torch.cuda.synchronize()
        stats = FrameStats(self.frame_index, k, self.map.n, self.map.capacity, is_key, sizes, float(self.loss.item()),
                           ev0.elapsed_time(ev1), 1e3 * (time.perf_counter() - t0), fused.get("ms", 0.0),
                           fused.get("blocks", 0), fused.get("touched", 0), fused.get("updated", 0))
        self.frame_index += 1
        return stats


def save_stream(opt: "StreamingOptimizer", path: str) -> None:
    """Checkpoint of the loop: the map with its Adam state (flat binary,
    checkpoint.py) at ``path``, and at ``path + ".state.npz"`` the position in
    the sequence, the keyframes' positions, the view sampler's state and the
    TSDF grid."""
    import json

    from . import checkpoint
    m = opt.map.model
    torch.cuda.synchronize()
    checkpoint.save_map(path, m.flat, m.m, m.v, m.n, opt.map.sh_degree, opt.step, opt.map.n)
    meta = {"frame_index": opt.frame_index, "step": opt.step, "novelty": opt.novelty,
            "rng": opt.rng.bit_generator.state, "n_live": int(opt.map.n), "n_slots": int(m.n),
            "map_bytes": os.path.getsize(path)}
    arrays = {"meta": np.frombuffer(json.dumps(meta).encode(), np.uint8),
              "keyframe_ids": np.asarray(opt.keyframe_ids, np.int64)}
    if opt.tsdf is not None:
        st = opt.tsdf.state()
        arrays.update({f"tsdf_{k}": np.asarray(v) for k, v in st.items()})
    tmp = f"{path}.state.tmp{os.getpid()}.npz"
    np.savez(tmp, **arrays)
    os.replace(tmp, path + ".state.npz")


def load_stream(opt: "StreamingOptimizer", path: str, frames) -> None:
    """Resumes ``opt`` (built with the same camera, SH degree and options)
    from ``save_stream``'s files; ``frames(i) -> (rgb, depth, pose)`` gives
    frame i of the sequence, for the keyframes' images."""
    import json

    from . import checkpoint
    d = checkpoint.load_map(path)
    if d["sh_degree"] != opt.map.sh_degree:
        raise ValueError("checkpoint SH degree differs from the optimizer's")
    with np.load(path + ".state.npz") as f:
        st = {k: f[k] for k in f.files}
    meta = json.loads(bytes(st["meta"]).decode())
    if meta["novelty"] != opt.novelty:
        raise ValueError(f"checkpoint of a {meta['novelty']!r} loop, the optimizer uses {opt.novelty!r}")
    # the map file and the state file are renamed into place one after the
    # other: a crash between the two leaves a pair from different steps
    mine = {"step": d["step"], "n_live": d["n_live"], "n_slots": d["n_slots"], "map_bytes": os.path.getsize(path)}
    theirs = {k: meta.get(k) for k in mine}
    if mine != theirs:
        raise ValueError(f"map file and state file are from different checkpoints: {mine} vs {theirs}")
    opt.map = GrowingMap(opt.map.sh_degree, d["n_slots"], opt.map.device)
    m = opt.map.model
    for dst, key in ((m.flat, "flat"), (m.m, "m"), (m.v, "v")):
        dst.copy_(torch.from_numpy(d[key]).to(dst.device))
    opt.map.n = d["n_live"]
    opt.step = d["step"]
    opt.frame_index = int(meta["frame_index"])
    opt.rng.bit_generator.state = meta["rng"]
    dev = m.flat.device
    opt.keyframes, opt.keyframe_ids = [], []
    for i in st["keyframe_ids"].tolist():
        rgb, depth, pose = frames(int(i))
        opt.keyframes.append(Keyframe(opt.cam, abi.make_viewmat(pose.R, pose.t),
                                      torch.as_tensor(np.ascontiguousarray(np.transpose(rgb, (2, 0, 1)),
                                                                           np.float32), device=dev),
                                      torch.as_tensor(np.ascontiguousarray(depth, np.float32), device=dev)))
        opt.keyframe_ids.append(int(i))
    if opt.tsdf is not None:
        opt.tsdf.load_state({k[5:]: v for k, v in st.items() if k.startswith("tsdf_")})
    torch.cuda.synchronize()


@dataclasses.dataclass
class GlobalStats:
    epochs: int
    keyframes: int
    steps: int
    view_iterations: int
    gpu_ms: float
    loss_first: float   # summed loss of the first batched step
    loss_last: float    # summed loss of the last batched step

    @property
    def ms_per_view_iteration(self) -> float:
        return self.gpu_ms / max(self.view_iterations, 1)


def global_optimize(opt: StreamingOptimizer, epochs: int = 2, views_per_step: int = 16,
                    rng_seed: int = 0) -> GlobalStats:
    """Offline optimisation over the keyframe list after the sequence (the
    paper's global optimisation, Sec. III-B.3 / IV): each epoch visits every
    keyframe once in a random order, ``views_per_step`` keyframes per batched
    iteration (gs_train_step_batched: the loss summed over them, one Adam
    step)."""
    rng = np.random.default_rng(rng_seed)
    kfs = opt.keyframes
    if not kfs:
        return GlobalStats(0, 0, 0, 0, 0.0, float("nan"), float("nan"))
    V = max(1, min(int(views_per_step), len(kfs), 16))
    H, W = opt.cam.height, opt.cam.width
    dev = opt.map.model.flat.device
    extra = V - len(opt.color)
    for _ in range(max(0, extra)):  # output slots for the larger batches
        opt.color.append(torch.empty((3, H, W), device=dev))
        opt.depth.append(torch.empty((H, W), device=dev))
        opt.alpha.append(torch.empty((H, W), device=dev))
        opt.dLdc.append(torch.empty((3, H, W), device=dev))
        opt.dLdd.append(torch.empty((H, W), device=dev))
    m = opt.map.model
    g = m.gaussians()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = views = 0
    first = None
    ev0.record()
    for _ in range(epochs):
        perm = rng.permutation(len(kfs))
        for s0 in range(0, len(kfs), V):
            batch = [kfs[i] for i in perm[s0:s0 + V]]
            n = len(batch)
            opt.step += 1
            abi.gs_train_step_batched(opt.ctx.handle, g, [opt.cam_s] * n, [k.view for k in batch], opt.rcfg,
                                      [k.rgb for k in batch], [k.depth for k in batch], opt.w_color, opt.w_depth,
                                      opt.loss, m.flat, m.m, m.v, opt.acfg, opt.step)
            if first is None:
                first = float(opt.loss.item())
            steps += 1
            views += n
    ev1.record()
    torch.cuda.synchronize()
    return GlobalStats(epochs, len(kfs), steps, views, ev0.elapsed_time(ev1), first, float(opt.loss.item()))
