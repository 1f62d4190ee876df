"""PyTorch-facing layer over the C ABI: device memory, streams, autograd.

* ``GaussianModel``   one flat float32 CUDA buffer holding the parameters in
                      the ABI's flat layout (means | log_scales | quats |
                      opacity_logits | sh), its gradient buffer and the Adam
                      moments, with per-array views.
* ``Trainer``         one optimisation iteration of GSFusion's online
                      optimisation (Sec. III-B.3) through the ABI:
                      gs_render_fwd -> gs_loss_l1 -> gs_render_bwd -> gs_adam_step.
* ``BatchedTrainer``  the same iteration over several views of one map in
                      one batched pass (one Adam step on the summed loss).
* ``render``          a torch.autograd.Function around gs_render_fwd /
                      gs_render_bwd (gradients for every parameter array and,
                      through a zero pose twist, the camera pose).

PyTorch is used for allocation and stream handles only; every arithmetic step
runs in libgsplat's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import abi

PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


def n_sh(deg: int) -> int:
    return (deg + 1) ** 2


def flat_sizes(n: int, deg: int):
    K = n_sh(deg)
    return [3 * n, 3 * n, 4 * n, n, 3 * K * n]


def _views(flat: torch.Tensor, n: int, deg: int) -> dict:
    K = n_sh(deg)
    shapes = [(n, 3), (n, 3), (n, 4), (n,), (n, K, 3)]
    out, off = {}, 0
    for name, size, shape in zip(PARAM_NAMES, flat_sizes(n, deg), shapes):
        out[name] = flat[off:off + size].view(shape)
        off += size
    return out


class GaussianModel:
    """Gaussian map in one flat buffer (plus gradient and Adam moments)."""

    def __init__(self, params: dict, device="cuda"):
        deg = int(params["sh_degree"])
        n = int(np.asarray(params["means"]).shape[0])
        self.n, self.sh_degree = n, deg
        total = sum(flat_sizes(n, deg))
        host = np.concatenate([np.asarray(params[k], np.float32).ravel() for k in PARAM_NAMES]) if n else \
            np.zeros(0, np.float32)
        assert host.size == total
        self.flat = torch.from_numpy(host).to(device)
        self.grad = torch.zeros_like(self.flat)
        self.m = torch.zeros_like(self.flat)
        self.v = torch.zeros_like(self.flat)
        self.p = _views(self.flat, n, deg)
        self.g = _views(self.grad, n, deg)

    def gaussians(self) -> abi.gs_gaussians:
        p = self.p
        return abi.make_gaussians(p["means"], p["log_scales"], p["quats"], p["opacity_logits"], p["sh"],
                                  self.sh_degree)

    def grads(self) -> abi.gs_grads:
        g = self.g
        return abi.make_grads(g["means"], g["log_scales"], g["quats"], g["opacity_logits"], g["sh"])

    def numpy_params(self) -> dict:
        out = {k: v.detach().cpu().numpy().copy() for k, v in self.p.items()}
        out["sh_degree"] = self.sh_degree
        return out


def camera_struct(cam) -> abi.gs_camera:
    return abi.make_camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)


def save_trainer(tr, path: str) -> None:
    """Checkpoint of a trainer's map, Adam moments and step (checkpoint.py)."""
    from . import checkpoint
    m = tr.model
    torch.cuda.synchronize()
    checkpoint.save_map(path, m.flat, m.m, m.v, m.n, m.sh_degree, tr.step_count)


def nonfinite_params(tr) -> int:
    """Number of NaN / +-Inf values among a trainer's parameters."""
    return abi.gs_count_nonfinite(tr.ctx.handle, tr.model.flat)


def load_trainer(tr, path: str) -> None:
    """Resumes a trainer from ``save_trainer``'s file: the map must have the
    same size and SH degree; the context's device Adam step is set too."""
    from . import checkpoint
    d = checkpoint.load_map(path)
    m = tr.model
    if d["n_slots"] != m.n or d["sh_degree"] != m.sh_degree:
        raise ValueError(f"checkpoint holds {d['n_slots']} Gaussians of SH degree {d['sh_degree']}, "
                         f"the trainer {m.n} of degree {m.sh_degree}")
    for dst, key in ((m.flat, "flat"), (m.m, "m"), (m.v, "v")):
        dst.copy_(torch.from_numpy(d[key]).to(dst.device))
    tr.step_count = d["step"]
    abi.gs_ctx_set_adam_step(tr.ctx.handle, d["step"])
    torch.cuda.synchronize()


class Context:
    """Owns one gs_ctx handle."""

    def __init__(self, device: int = 0, pair_capacity: int = 0):
        self.handle = abi.gs_ctx_create(device, pair_capacity)

    def close(self):
        if self.handle:
            abi.gs_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self) -> dict:
        return abi.gs_get_stats(self.handle)


class Trainer:
    """One view, one map: fwd + L1 loss + bwd + Adam per ``step``.

    ``one_call`` (default) runs the whole iteration as gs_train_step (loss in
    the compositing epilogue, backward fused with Adam; the rendered images
    stay unwritten).  Otherwise ``fused`` runs gs_render_fwd + gs_loss_l1 +
    gs_render_bwd_adam (no gradient buffer), or, with fused=False,
    gs_render_bwd into the model's gradient buffer followed by gs_adam_step
    (which clears it)."""

    def __init__(self, model: GaussianModel, cam, R, t, raster_cfg=None, adam_cfg=None, w_color=0.8, w_depth=0.2,
                 ctx: Context | None = None, device: int = 0, fused: bool = True, one_call: bool = True):
        self.fused = fused
        self.one_call = one_call and fused
        self.model = model
        self.ctx = ctx or Context(device)
        self.cam = camera_struct(cam)
        self.view = abi.make_viewmat(R, t)
        self.rcfg = raster_cfg or abi.raster_cfg()
        self.acfg = adam_cfg or abi.adam_cfg(zero_grads=1)
        self.w_color, self.w_depth = float(w_color), float(w_depth)
        H, W = cam.height, cam.width
        dev = model.flat.device
        self.color = torch.empty((3, H, W), device=dev)
        self.depth = torch.empty((H, W), device=dev)
        self.alpha = torch.empty((H, W), device=dev)
        self.dLdc = torch.empty((3, H, W), device=dev)
        self.dLdd = torch.empty((H, W), device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.step_count = 0
        self._g = model.gaussians()
        self._gr = model.grads()

    def forward(self, stream=None):
        abi.gs_render_fwd(self.ctx.handle, self._g, self.cam, self.view, self.rcfg, self.color, self.depth,
                          self.alpha, stream)

    def step(self, target_rgb: torch.Tensor, target_depth: torch.Tensor, stream=None):
        """One iteration; the loss of the rendered image stays on the device in
        ``self.loss``.  Gradients are cleared by the Adam kernel."""
        h = self.ctx.handle
        m = self.model
        if self.one_call:
            self.step_count += 1
            abi.gs_train_step(h, self._g, self.cam, self.view, self.rcfg, target_rgb, target_depth, self.w_color,
                              self.w_depth, self.loss, m.flat, m.m, m.v, self.acfg, self.step_count, stream)
            return self.loss
        self.forward(stream)
        abi.gs_loss_l1(h, self.cam, self.color, self.depth, target_rgb, target_depth, self.w_color, self.w_depth,
                       self.loss, self.dLdc, self.dLdd, stream)
        self.step_count += 1
        if self.fused:
            abi.gs_render_bwd_adam(h, self._g, self.cam, self.view, self.rcfg, self.dLdc, self.dLdd, None, m.flat, m.m,
                                   m.v, self.acfg, self.step_count, None, stream)
        else:
            abi.gs_render_bwd(h, self._g, self.cam, self.view, self.rcfg, self.dLdc, self.dLdd, None, self._gr, None,
                              stream)
            abi.gs_adam_step(h, m.flat, m.grad, m.m, m.v, m.n, m.sh_degree, self.acfg, self.step_count, stream)
        return self.loss

    def _step_device_counter(self, target_rgb, target_depth, stream=None):
        # one iteration whose every argument is fixed: the Adam step comes from
        # the context's device counter (step = 0), so it can be graph-captured
        h = self.ctx.handle
        m = self.model
        if self.one_call:
            abi.gs_train_step(h, self._g, self.cam, self.view, self.rcfg, target_rgb, target_depth, self.w_color,
                              self.w_depth, self.loss, m.flat, m.m, m.v, self.acfg, 0, stream)
            return
        self.forward(stream)
        abi.gs_loss_l1(h, self.cam, self.color, self.depth, target_rgb, target_depth, self.w_color, self.w_depth,
                       self.loss, self.dLdc, self.dLdd, stream)
        abi.gs_render_bwd_adam(h, self._g, self.cam, self.view, self.rcfg, self.dLdc, self.dLdd, None, m.flat, m.m,
                               m.v, self.acfg, 0, None, stream)

    def autotune(self, reps: int = 5) -> list:
        """Pick the fastest tile shape for this view (gs_autotune)."""
        return abi.gs_autotune(self.ctx.handle, self._g, [self.cam], [self.view], self.rcfg, reps)

    def capture(self, target_rgb: torch.Tensor, target_depth: torch.Tensor, pair_headroom: float = 1.5):
        """Record one iteration into a CUDA graph (``replay`` runs it).

        Switches the context to no-sync mode with the pair buffers reserved at
        ``pair_headroom`` times the current pair count; the graph reads the
        targets from ``target_rgb`` / ``target_depth`` (copy new frames into
        them).  Runs one eager no-sync iteration first (a real step)."""
        assert self.fused, "graph capture uses the fused backward + Adam"
        h = self.ctx.handle
        self.forward()
        torch.cuda.synchronize()
        pairs = abi.gs_get_stats(h)["n_pairs"]
        H, W = self.cam.height, self.cam.width
        abi.gs_ctx_reserve(h, self.model.n, H * W, int(pairs * pair_headroom) + 4096)
        abi.gs_ctx_set_sync(h, False)
        abi.gs_ctx_set_adam_step(h, self.step_count)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self._step_device_counter(target_rgb, target_depth)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.step_count += 1
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._step_device_counter(target_rgb, target_depth)
        return self.graph

    def replay(self):
        """One captured iteration; the loss stays on the device in ``self.loss``."""
        self.graph.replay()
        self.step_count += 1
        return self.loss

    def capture_from_host(self, host_rgb: torch.Tensor, host_depth: torch.Tensor, host_loss: torch.Tensor,
                          buffers) -> list:
        """Record a double-buffered host-to-host loop as two CUDA graphs.
        Graph b runs the iteration on the device targets buffers[b] = (rgb
        [3, H, W], depth [H, W]) and copies the loss into pinned host_loss
        [1], while a forked branch uploads the next frame from pinned host
        memory (host_rgb, host_depth) into buffers[1 - b]; replaying graph 0,
        1, 0, ... is one step each (the first frame is uploaded into
        buffers[0] before the first replay; refill the host buffers between
        replays once the previous replay has finished).  Call after
        ``capture`` (no-sync mode, buffers reserved)."""
        if not (host_rgb.is_pinned() and host_depth.is_pinned() and host_loss.is_pinned()):
            raise ValueError("host buffers must be pinned")
        side = torch.cuda.Stream()
        graphs = []
        for b in range(2):
            cur_rgb, cur_dep = buffers[b]
            nxt_rgb, nxt_dep = buffers[1 - b]
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                main = torch.cuda.current_stream()
                side.wait_stream(main)
                with torch.cuda.stream(side):
                    nxt_rgb.copy_(host_rgb, non_blocking=True)
                    nxt_dep.copy_(host_depth, non_blocking=True)
                self._step_device_counter(cur_rgb, cur_dep)
                host_loss.copy_(self.loss, non_blocking=True)
                main.wait_stream(side)
            graphs.append(g)
        return graphs

    def check_capacity(self):
        """Raises GsError(GS_ERR_CAPACITY) if a no-sync pass dropped pairs."""
        abi.gs_sync_status(self.ctx.handle)

    def save(self, path: str) -> None:
        save_trainer(self, path)

    def load(self, path: str) -> None:
        load_trainer(self, path)

    def nonfinite(self) -> int:
        return nonfinite_params(self)


class BatchedTrainer:
    """Several views, one map: one batched iteration per ``step``.

    ``views`` is a list of (camera, R_cw, t_cw).  A step renders every view
    (gs_render_fwd_batched), scores it (gs_loss_l1_batched: the sum of the
    per-view losses) and runs the backward pass of all views fused with one
    Adam step on the summed gradient (gs_render_bwd_adam_batched).
    ``step_sequential`` computes the same iteration with the single-view
    calls, one view at a time (gradients accumulated, then gs_adam_step)."""

    def __init__(self, model: GaussianModel, views, raster_cfg=None, adam_cfg=None, w_color=0.8, w_depth=0.2,
                 ctx: Context | None = None, device: int = 0, one_call: bool = True):
        self.one_call = one_call
        self.model = model
        self.ctx = ctx or Context(device)
        self.cam_list = list(c for c, _, _ in views)
        self.cams = [camera_struct(c) for c, _, _ in views]
        self.vms = [abi.make_viewmat(R, t) for _, R, t in views]
        self.rcfg = raster_cfg or abi.raster_cfg()
        self.acfg = adam_cfg or abi.adam_cfg(zero_grads=1)
        self.w_color, self.w_depth = float(w_color), float(w_depth)
        dev = model.flat.device
        self.color = [torch.empty((3, c.height, c.width), device=dev) for c in self.cam_list]
        self.depth = [torch.empty((c.height, c.width), device=dev) for c in self.cam_list]
        self.alpha = [torch.empty((c.height, c.width), device=dev) for c in self.cam_list]
        self.dLdc = [torch.empty((3, c.height, c.width), device=dev) for c in self.cam_list]
        self.dLdd = [torch.empty((c.height, c.width), device=dev) for c in self.cam_list]
        self.loss = torch.zeros(1, device=dev)
        self.loss_views = torch.zeros(len(views), device=dev)  # per-view losses of step_sequential
        self.step_count = 0
        self._g = model.gaussians()
        self._gr = model.grads()

    @property
    def n_views(self) -> int:
        return len(self.cams)

    @property
    def n_pixels(self) -> int:
        return sum(c.width * c.height for c in self.cam_list)

    def forward(self, stream=None):
        abi.gs_render_fwd_batched(self.ctx.handle, self._g, self.cams, self.vms, self.rcfg, self.color, self.depth,
                                  self.alpha, stream)

    def _iteration(self, targets_rgb, targets_depth, step, stream=None):
        h = self.ctx.handle
        m = self.model
        if self.one_call:  # gs_train_step_batched (the rendered images are written too)
            abi.gs_train_step_batched(h, self._g, self.cams, self.vms, self.rcfg, targets_rgb, targets_depth,
                                      self.w_color, self.w_depth, self.loss, m.flat, m.m, m.v, self.acfg, step,
                                      self.color, self.depth, self.alpha, stream)
            return
        self.forward(stream)
        abi.gs_loss_l1_batched(h, self.cams, self.color, self.depth, targets_rgb, targets_depth, self.w_color,
                               self.w_depth, self.loss, self.dLdc, self.dLdd, stream)
        abi.gs_render_bwd_adam_batched(h, self._g, self.cams, self.vms, self.rcfg, self.dLdc, self.dLdd, None, m.flat,
                                       m.m, m.v, self.acfg, step, None, stream)

    def step(self, targets_rgb, targets_depth, stream=None):
        """One batched iteration; the summed loss stays on the device in ``self.loss``.
        ``one_call`` (default) runs it as gs_train_step_batched, otherwise as
        gs_render_fwd_batched + gs_loss_l1_batched + gs_render_bwd_adam_batched."""
        self.step_count += 1
        self._iteration(targets_rgb, targets_depth, self.step_count, stream)
        return self.loss

    def step_sequential(self, targets_rgb, targets_depth, stream=None):
        """The same iteration view by view with the single-view calls: per view
        gs_render_fwd, gs_loss_l1 and gs_render_bwd (gradients accumulate in
        the model's gradient buffer), then one gs_adam_step, which clears it.
        Returns the per-view losses (device [V]; their sum is the batched loss)."""
        h = self.ctx.handle
        m = self.model
        for v in range(self.n_views):
            abi.gs_render_fwd(h, self._g, self.cams[v], self.vms[v], self.rcfg, self.color[v], self.depth[v],
                              self.alpha[v], stream)
            abi.gs_loss_l1(h, self.cams[v], self.color[v], self.depth[v], targets_rgb[v], targets_depth[v],
                           self.w_color, self.w_depth, self.loss_views[v:v + 1], self.dLdc[v], self.dLdd[v], stream)
            abi.gs_render_bwd(h, self._g, self.cams[v], self.vms[v], self.rcfg, self.dLdc[v], self.dLdd[v], None,
                              self._gr, None, stream)
        self.step_count += 1
        abi.gs_adam_step(h, m.flat, m.grad, m.m, m.v, m.n, m.sh_degree, self.acfg, self.step_count, stream)
        return self.loss_views

    def autotune(self, reps: int = 5) -> list:
        """Pick the fastest tile shape for these views (gs_autotune); returns
        the milliseconds per pass of each candidate shape."""
        return abi.gs_autotune(self.ctx.handle, self._g, self.cams, self.vms, self.rcfg, reps)

    def _sequential_device_counter(self, targets_rgb, targets_depth):
        h = self.ctx.handle
        m = self.model
        for v in range(self.n_views):
            abi.gs_render_fwd(h, self._g, self.cams[v], self.vms[v], self.rcfg, self.color[v], self.depth[v],
                              self.alpha[v])
            abi.gs_loss_l1(h, self.cams[v], self.color[v], self.depth[v], targets_rgb[v], targets_depth[v],
                           self.w_color, self.w_depth, self.loss_views[v:v + 1], self.dLdc[v], self.dLdd[v])
            abi.gs_render_bwd(h, self._g, self.cams[v], self.vms[v], self.rcfg, self.dLdc[v], self.dLdd[v], None,
                              self._gr, None)
        abi.gs_adam_step(h, m.flat, m.grad, m.m, m.v, m.n, m.sh_degree, self.acfg, 0)

    def capture_sequential(self, targets_rgb, targets_depth, pair_headroom: float = 1.5):
        """Record ``step_sequential`` (one view at a time, then one Adam step on
        the device step counter) into a CUDA graph (``replay`` runs it): the
        strongest form of the view-by-view comparison."""
        h = self.ctx.handle
        pairs = 0
        for v in range(self.n_views):
            abi.gs_render_fwd(h, self._g, self.cams[v], self.vms[v], self.rcfg)
            torch.cuda.synchronize()
            pairs = max(pairs, abi.gs_get_stats(h)["n_pairs"])
        npx = max(c.width * c.height for c in self.cam_list)
        abi.gs_ctx_reserve(h, self.model.n, npx, int(pairs * pair_headroom) + 4096)
        abi.gs_ctx_set_sync(h, False)
        abi.gs_ctx_set_adam_step(h, self.step_count)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self._sequential_device_counter(targets_rgb, targets_depth)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.step_count += 1
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._sequential_device_counter(targets_rgb, targets_depth)
        return self.graph

    def capture(self, targets_rgb, targets_depth, pair_headroom: float = 1.5):
        """Record one batched iteration into a CUDA graph (``replay`` runs it),
        as Trainer.capture does for one view."""
        h = self.ctx.handle
        self.forward()
        torch.cuda.synchronize()
        pairs = abi.gs_get_stats(h)["n_pairs"]
        abi.gs_ctx_reserve(h, self.model.n * self.n_views, self.n_pixels, int(pairs * pair_headroom) + 4096)
        abi.gs_ctx_set_sync(h, False)
        abi.gs_ctx_set_adam_step(h, self.step_count)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self._iteration(targets_rgb, targets_depth, 0)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.step_count += 1
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._iteration(targets_rgb, targets_depth, 0)
        return self.graph

    def replay(self):
        self.graph.replay()
        self.step_count += 1
        return self.loss

    def check_capacity(self):
        abi.gs_sync_status(self.ctx.handle)

    def save(self, path: str) -> None:
        save_trainer(self, path)

    def load(self, path: str) -> None:
        load_trainer(self, path)

    def nonfinite(self) -> int:
        return nonfinite_params(self)


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(actx, means, log_scales, quats, opacity_logits, sh, pose_xi, meta):
        ctx, cam, view, rcfg, deg = meta
        g = abi.make_gaussians(means.contiguous(), log_scales.contiguous(), quats.contiguous(),
                               opacity_logits.contiguous(), sh.contiguous(), deg)
        H, W = cam.height, cam.width
        color = torch.empty((3, H, W), device=means.device)
        depth = torch.empty((H, W), device=means.device)
        alpha = torch.empty((H, W), device=means.device)
        abi.gs_render_fwd(ctx.handle, g, cam, view, rcfg, color, depth, alpha)
        actx.meta = meta
        actx.token = abi.gs_state_token(ctx.handle)
        actx.save_for_backward(means, log_scales, quats, opacity_logits, sh)
        actx.pose_device = pose_xi.device if pose_xi is not None else None
        return color, depth, alpha

    @staticmethod
    def backward(actx, gc, gd, ga):
        ctx, cam, view, rcfg, deg = actx.meta
        means, log_scales, quats, opacity_logits, sh = actx.saved_tensors
        g = abi.make_gaussians(means.contiguous(), log_scales.contiguous(), quats.contiguous(),
                               opacity_logits.contiguous(), sh.contiguous(), deg)
        grads = [torch.zeros_like(t) for t in (means, log_scales, quats, opacity_logits, sh)]
        gp = torch.zeros(6, device=means.device)
        zero = torch.zeros((cam.height, cam.width), device=means.device)
        gc = gc.contiguous() if gc is not None else torch.zeros((3, cam.height, cam.width), device=means.device)
        gd = gd.contiguous() if gd is not None else zero
        ga = ga.contiguous() if ga is not None else None
        if abi.gs_state_token(ctx.handle) != actx.token:
            # another forward pass ran on this context since (e.g. a second
            # render of the same map at another pose): recompute this one's
            # state from the saved inputs before differentiating it
            abi.gs_render_fwd(ctx.handle, g, cam, view, rcfg, None, None, None)
        try:
            abi.gs_render_bwd(ctx.handle, g, cam, view, rcfg, gc, gd, ga, abi.make_grads(*grads), gp)
        except abi.GsError as e:
            if e.status != abi.GS_ERR_STATE:
                raise
            # inputs that were not contiguous were copied, so the arrays differ
            # from the forward pass's: recompute the state from these copies
            abi.gs_render_fwd(ctx.handle, g, cam, view, rcfg, None, None, None)
            abi.gs_render_bwd(ctx.handle, g, cam, view, rcfg, gc, gd, ga, abi.make_grads(*grads), gp)
        pose_grad = gp.to(actx.pose_device) if actx.pose_device is not None else None
        return (*grads, pose_grad, None)


def render(ctx: Context, params: dict, sh_degree: int, cam, R, t, raster_cfg=None, pose_xi=None):
    """Differentiable render of (colour [3, H, W], depth [H, W], alpha [H, W]).

    ``params`` maps the five parameter names to CUDA float32 tensors.  If
    ``pose_xi`` (a zero 6-vector with requires_grad) is given, its gradient is
    dL/dxi of the left perturbation exp(xi^) T_CW at xi = 0."""
    cam_s = camera_struct(cam)
    view = abi.make_viewmat(R, t)
    rcfg = raster_cfg or abi.raster_cfg()
    meta = (ctx, cam_s, view, rcfg, int(sh_degree))
    return _Render.apply(params["means"], params["log_scales"], params["quats"], params["opacity_logits"],
                         params["sh"], pose_xi, meta)
