"""ctypes binding of libgsplat (include/gsplat.h): argument marshalling only.

Every function here has the name of the C entry point it calls and takes
torch CUDA tensors (or plain ints / floats) where the C function takes device
pointers.  No computation happens in Python: every step of the path runs in
the library's kernels.  Loading fails loudly when libgsplat.so is missing;
there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgsplat.so")
CHECKED_LIB_PATH = os.path.join(HERE, "libgsplat_checked.so")  # bounds-checked build (gs_bounds_checked)

GS_OK = 0
STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_CUDA", 3: "GS_ERR_CAPACITY", 4: "GS_ERR_NONFINITE",
                5: "GS_ERR_BOUNDS", 6: "GS_ERR_TIMEOUT", 7: "GS_ERR_OOM", 8: "GS_ERR_STATE"}


GS_ERR_INVALID_ARG, GS_ERR_CUDA, GS_ERR_CAPACITY, GS_ERR_OOM, GS_ERR_STATE = 1, 2, 3, 7, 8


class GsError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class gs_camera(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32)]


class gs_viewmat(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3)]


class gs_gaussians(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64), ("sh_degree", C.c_int32)]


class gs_grads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p)]


class gs_raster_cfg(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("batch", C.c_int32), ("bg", C.c_float * 3),
                ("near_z", C.c_float), ("alpha_max", C.c_float), ("alpha_min", C.c_float), ("t_eps", C.c_float),
                ("dilation", C.c_float)]


class gs_adam_cfg(C.Structure):
    _fields_ = [("lr_means", C.c_float), ("lr_log_scales", C.c_float), ("lr_quats", C.c_float),
                ("lr_opacity", C.c_float), ("lr_sh_dc", C.c_float), ("lr_sh_rest", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float), ("zero_grads", C.c_int32)]


class gs_stats(C.Structure):
    _fields_ = [("n_pairs", C.c_int64), ("pair_capacity", C.c_int64), ("kernel_launches", C.c_int64),
                ("n_tiles", C.c_int64), ("evals_blended", C.c_int64), ("evals_tiled", C.c_int64)]


class gs_alu_peaks(C.Structure):
    _fields_ = [("fma_tflops", C.c_double), ("ex2_gops", C.c_double), ("fma_sm_mhz", C.c_double),
                ("ex2_sm_mhz", C.c_double), ("fma_per_sm_clk", C.c_double), ("ex2_per_sm_clk", C.c_double),
                ("fma_ms", C.c_double), ("ex2_ms", C.c_double), ("num_sms", C.c_int32)]


class gs_tsdf_grid(C.Structure):
    _fields_ = [("keys", C.c_void_p), ("slots", C.c_void_p), ("stamps", C.c_void_p), ("voxels", C.c_void_p),
                ("claims", C.c_void_p), ("touched", C.c_void_p), ("counters", C.c_void_p),
                ("table_size", C.c_int64), ("capacity", C.c_int64), ("voxel_size", C.c_float),
                ("truncation", C.c_float), ("max_weight", C.c_float), ("fusion", C.c_int32)]


STAGES = ("project_fwd", "depth_sort", "duplicate", "pair_sort", "ranges", "raster_fwd", "loss", "raster_bwd",
          "project_bwd", "adam")


P = C.c_void_p
PP = C.POINTER(C.c_void_p)  # host array of device pointers
EXPORTS = {
    "gs_ctx_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int64]),
    "gs_ctx_destroy": (C.c_int, [P]),
    "gs_last_error": (C.c_char_p, [P]),
    "gs_ctx_reserve": (C.c_int, [P, C.c_int64, C.c_int64, C.c_int64]),
    "gs_ctx_set_sync": (C.c_int, [P, C.c_int]),
    "gs_ctx_set_adam_step": (C.c_int, [P, C.c_int64]),
    "gs_ctx_set_tile_order": (C.c_int, [P, C.c_int]),
    "gs_ctx_set_persistent": (C.c_int, [P, C.c_int]),
    "gs_sync_status": (C.c_int, [P, P]),
    "gs_get_stats": (C.c_int, [P, C.POINTER(gs_stats)]),
    "gs_raster_cfg_default": (C.c_int, [C.POINTER(gs_raster_cfg)]),
    "gs_adam_cfg_default": (C.c_int, [C.POINTER(gs_adam_cfg)]),
    "gs_render_fwd": (C.c_int, [P, C.POINTER(gs_gaussians), C.POINTER(gs_camera), C.POINTER(gs_viewmat),
                                C.POINTER(gs_raster_cfg), P, P, P, P]),
    "gs_render_bwd": (C.c_int, [P, C.POINTER(gs_gaussians), C.POINTER(gs_camera), C.POINTER(gs_viewmat),
                                C.POINTER(gs_raster_cfg), P, P, P, C.POINTER(gs_grads), P, P]),
    "gs_render_bwd_adam": (C.c_int, [P, C.POINTER(gs_gaussians), C.POINTER(gs_camera), C.POINTER(gs_viewmat),
                                     C.POINTER(gs_raster_cfg), P, P, P, P, P, P, C.POINTER(gs_adam_cfg), C.c_int64,
                                     P, P]),
    "gs_loss_l1": (C.c_int, [P, C.POINTER(gs_camera), P, P, P, P, C.c_float, C.c_float, P, P, P, P]),
    "gs_adam_step": (C.c_int, [P, P, P, P, P, C.c_int64, C.c_int32, C.POINTER(gs_adam_cfg), C.c_int64, P]),
    "gs_bin_tiles": (C.c_int, [P, C.c_int64, P, P, P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P, P, P, C.c_int64,
                               C.POINTER(C.c_int64), P]),
    "gs_get_projection": (C.c_int, [P, P, P, P, P, P, P, P]),
    "gs_loss_l1_noalloc": (C.c_int, [C.POINTER(gs_camera), P, P, P, P, C.c_float, C.c_float, P, P, P, P]),
    "gs_render_fwd_batched": (C.c_int, [P, C.POINTER(gs_gaussians), C.c_int32, C.POINTER(gs_camera),
                                        C.POINTER(gs_viewmat), C.POINTER(gs_raster_cfg), PP, PP, PP, P]),
    "gs_render_bwd_batched": (C.c_int, [P, C.POINTER(gs_gaussians), C.c_int32, C.POINTER(gs_camera),
                                        C.POINTER(gs_viewmat), C.POINTER(gs_raster_cfg), PP, PP, PP,
                                        C.POINTER(gs_grads), P, P]),
    "gs_render_bwd_adam_batched": (C.c_int, [P, C.POINTER(gs_gaussians), C.c_int32, C.POINTER(gs_camera),
                                             C.POINTER(gs_viewmat), C.POINTER(gs_raster_cfg), PP, PP, PP, P, P, P,
                                             C.POINTER(gs_adam_cfg), C.c_int64, P, P]),
    "gs_loss_l1_batched": (C.c_int, [P, C.c_int32, C.POINTER(gs_camera), PP, PP, PP, PP, C.c_float, C.c_float, P,
                                     PP, PP, P]),
    "gs_train_step": (C.c_int, [P, C.POINTER(gs_gaussians), C.POINTER(gs_camera), C.POINTER(gs_viewmat),
                                C.POINTER(gs_raster_cfg), P, P, C.c_float, C.c_float, P, P, P, P,
                                C.POINTER(gs_adam_cfg), C.c_int64, P]),
    "gs_train_step_batched": (C.c_int, [P, C.POINTER(gs_gaussians), C.c_int32, C.POINTER(gs_camera),
                                        C.POINTER(gs_viewmat), C.POINTER(gs_raster_cfg), PP, PP, C.c_float,
                                        C.c_float, P, P, P, P, C.POINTER(gs_adam_cfg), C.c_int64, PP, PP, PP, P]),
    "gs_quadtree_leaves": (C.c_int, [P, P, C.c_int32, C.c_int32, C.c_float, C.c_int32, C.c_int32, P, C.c_int64,
                                     C.POINTER(C.c_int64), P]),
    "gs_seed_quadtree": (C.c_int, [P, P, P, P, C.c_float, C.POINTER(gs_camera), C.POINTER(gs_viewmat), C.c_int32,
                                   C.c_float, C.c_int32, C.c_int32, P, P, P, P, P, C.c_int64,
                                   C.POINTER(C.c_int64), P]),
    "gs_tsdf_integrate": (C.c_int, [P, C.POINTER(gs_tsdf_grid), P, C.POINTER(gs_camera), C.POINTER(gs_viewmat),
                                    C.c_uint32, C.c_int64, P]),
    "gs_tsdf_counters": (C.c_int, [P, C.POINTER(gs_tsdf_grid), C.POINTER(C.c_int64), P]),
    "gs_tsdf_rehash": (C.c_int, [P, C.POINTER(gs_tsdf_grid), C.POINTER(gs_tsdf_grid), P]),
    "gs_tsdf_query": (C.c_int, [P, C.POINTER(gs_tsdf_grid), P, C.c_int64, P, P, P]),
    "gs_seed_tsdf": (C.c_int, [P, P, P, C.POINTER(gs_tsdf_grid), C.POINTER(gs_camera), C.POINTER(gs_viewmat),
                               C.c_int32, C.c_float, C.c_int32, C.c_int32, P, P, P, P, P, C.c_int64,
                               C.POINTER(C.c_int64), P]),
    "gs_count_nonfinite": (C.c_int, [P, P, C.c_int64, C.POINTER(C.c_int64), P]),
    "gs_ctx_inject_alloc_failure": (C.c_int, [P, C.c_int32]),
    "gs_bounds_checked": (C.c_int, []),
    "gs_ctx_inject_bounds_fault": (C.c_int, [P]),
    "gs_autotune": (C.c_int, [P, C.POINTER(gs_gaussians), C.c_int32, C.POINTER(gs_camera), C.POINTER(gs_viewmat),
                              C.POINTER(gs_raster_cfg), C.c_int32, C.POINTER(C.c_float), P]),
    "gs_set_eval_counting": (C.c_int, [P, C.c_int]),
    "gs_set_profiling": (C.c_int, [P, C.c_int]),
    "gs_profile_read": (C.c_int, [P, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "gs_measure_alu_peaks": (C.c_int, [C.c_int, C.c_int32, C.POINTER(gs_alu_peaks)]),
    "gs_state_token": (C.c_int, [P, C.POINTER(C.c_uint64)]),
    "gs_get_tile_ranges": (C.c_int, [P, P, C.c_int64, P]),
    "gs_get_tile_order": (C.c_int, [P, P, C.c_int64, P]),
}

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libgsplat.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libgsplat.so not found at {path}; run __graft_entry__.build() first")
        lib = C.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _f32(t, name):
    if t is not None and t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    return _ptr(t)


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(ctx, status: int, where: str):
    if status != GS_OK:
        msg = load().gs_last_error(ctx).decode() if ctx else ""
        raise GsError(status, where, msg)


# ---------------------------------------------------------------------------
# struct builders
# ---------------------------------------------------------------------------
def make_camera(fx, fy, cx, cy, width, height) -> gs_camera:
    return gs_camera(float(fx), float(fy), float(cx), float(cy), int(width), int(height))


def make_viewmat(R, t) -> gs_viewmat:
    v = gs_viewmat()
    Rf = [float(x) for x in torch.as_tensor(R).reshape(-1).tolist()]
    tf = [float(x) for x in torch.as_tensor(t).reshape(-1).tolist()]
    v.R = (C.c_float * 9)(*Rf)
    v.t = (C.c_float * 3)(*tf)
    return v


def raster_cfg(**overrides) -> gs_raster_cfg:
    c = gs_raster_cfg()
    load().gs_raster_cfg_default(C.byref(c))
    for k, v in overrides.items():
        if k == "bg":
            c.bg = (C.c_float * 3)(*[float(x) for x in v])
        else:
            setattr(c, k, v)
    return c


def adam_cfg(**overrides) -> gs_adam_cfg:
    c = gs_adam_cfg()
    load().gs_adam_cfg_default(C.byref(c))
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


def make_gaussians(means, log_scales, quats, opacity_logits, sh, sh_degree: int) -> gs_gaussians:
    n = means.shape[0]
    return gs_gaussians(_f32(means, "means"), _f32(log_scales, "log_scales"), _f32(quats, "quats"),
                        _f32(opacity_logits, "opacity_logits"), _f32(sh, "sh"), int(n), int(sh_degree))


def make_grads(means, log_scales, quats, opacity_logits, sh) -> gs_grads:
    return gs_grads(_f32(means, "means"), _f32(log_scales, "log_scales"), _f32(quats, "quats"),
                    _f32(opacity_logits, "opacity_logits"), _f32(sh, "sh"))


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def gs_ctx_create(device: int = 0, pair_capacity: int = 0) -> int:
    h = C.c_void_p()
    st = load().gs_ctx_create(C.byref(h), int(device), int(pair_capacity))
    _check(None, st, "gs_ctx_create")
    return h.value


def gs_ctx_destroy(ctx: int) -> None:
    _check(None, load().gs_ctx_destroy(ctx), "gs_ctx_destroy")


def gs_last_error(ctx: int) -> str:
    return load().gs_last_error(ctx).decode()


def gs_ctx_reserve(ctx, n_gaussians=0, n_pixels=0, n_pairs=0):
    _check(ctx, load().gs_ctx_reserve(ctx, int(n_gaussians), int(n_pixels), int(n_pairs)), "gs_ctx_reserve")


def gs_ctx_set_sync(ctx, sync: bool):
    _check(ctx, load().gs_ctx_set_sync(ctx, int(bool(sync))), "gs_ctx_set_sync")


def gs_ctx_set_adam_step(ctx, step: int):
    _check(ctx, load().gs_ctx_set_adam_step(ctx, int(step)), "gs_ctx_set_adam_step")


def gs_ctx_set_tile_order(ctx, on: bool):
    _check(ctx, load().gs_ctx_set_tile_order(ctx, int(bool(on))), "gs_ctx_set_tile_order")


def gs_ctx_set_persistent(ctx, on: bool):
    _check(ctx, load().gs_ctx_set_persistent(ctx, int(bool(on))), "gs_ctx_set_persistent")


def gs_sync_status(ctx, stream=None):
    _check(ctx, load().gs_sync_status(ctx, _stream(stream)), "gs_sync_status")


def gs_get_stats(ctx) -> dict:
    s = gs_stats()
    _check(ctx, load().gs_get_stats(ctx, C.byref(s)), "gs_get_stats")
    return {k: getattr(s, k) for k, _ in gs_stats._fields_}


def gs_set_eval_counting(ctx, counting: bool):
    _check(ctx, load().gs_set_eval_counting(ctx, int(bool(counting))), "gs_set_eval_counting")


def gs_set_profiling(ctx, profiling: bool):
    _check(ctx, load().gs_set_profiling(ctx, int(bool(profiling))), "gs_set_profiling")


def gs_profile_read(ctx) -> dict:
    """{stage: (total ms, launches)} since profiling was switched on / last read."""
    ms = (C.c_double * len(STAGES))()
    cnt = (C.c_int64 * len(STAGES))()
    _check(ctx, load().gs_profile_read(ctx, ms, cnt), "gs_profile_read")
    return {s: (ms[i], cnt[i]) for i, s in enumerate(STAGES)}


def gs_render_fwd(ctx, gaussians: gs_gaussians, cam: gs_camera, view: gs_viewmat, cfg: gs_raster_cfg,
                  color=None, depth=None, alpha=None, stream=None):
    st = load().gs_render_fwd(ctx, C.byref(gaussians), C.byref(cam), C.byref(view), C.byref(cfg),
                              _f32(color, "color"), _f32(depth, "depth"), _f32(alpha, "alpha"), _stream(stream))
    _check(ctx, st, "gs_render_fwd")


def gs_render_bwd(ctx, gaussians, cam, view, cfg, dL_dcolor, dL_ddepth, dL_dalpha, grads: gs_grads,
                  dL_dpose=None, stream=None):
    st = load().gs_render_bwd(ctx, C.byref(gaussians), C.byref(cam), C.byref(view), C.byref(cfg),
                              _f32(dL_dcolor, "dL_dcolor"), _f32(dL_ddepth, "dL_ddepth"),
                              _f32(dL_dalpha, "dL_dalpha"), C.byref(grads), _f32(dL_dpose, "dL_dpose"),
                              _stream(stream))
    _check(ctx, st, "gs_render_bwd")


def gs_render_bwd_adam(ctx, gaussians, cam, view, cfg, dL_dcolor, dL_ddepth, dL_dalpha, params, m, v,
                       adam: gs_adam_cfg, step: int, dL_dpose=None, stream=None):
    st = load().gs_render_bwd_adam(ctx, C.byref(gaussians), C.byref(cam), C.byref(view), C.byref(cfg),
                                   _f32(dL_dcolor, "dL_dcolor"), _f32(dL_ddepth, "dL_ddepth"),
                                   _f32(dL_dalpha, "dL_dalpha"), _f32(params, "params"), _f32(m, "m"), _f32(v, "v"),
                                   C.byref(adam), int(step), _f32(dL_dpose, "dL_dpose"), _stream(stream))
    _check(ctx, st, "gs_render_bwd_adam")


def gs_loss_l1(ctx, cam, color, depth, target_rgb, target_depth, w_color, w_depth, loss, dL_dcolor, dL_ddepth,
               stream=None):
    st = load().gs_loss_l1(ctx, C.byref(cam), _f32(color, "color"), _f32(depth, "depth"),
                           _f32(target_rgb, "target_rgb"), _f32(target_depth, "target_depth"), float(w_color),
                           float(w_depth), _f32(loss, "loss"), _f32(dL_dcolor, "dL_dcolor"),
                           _f32(dL_ddepth, "dL_ddepth"), _stream(stream))
    _check(ctx, st, "gs_loss_l1")


def gs_loss_l1_noalloc(cam, color, depth, target_rgb, target_depth, w_color, w_depth, loss, dL_dcolor, dL_ddepth,
                       stream=None):
    """gs_loss_l1 for callers that must not allocate device memory (scratch
    comes from a fixed array inside the library; see include/gsplat.h)."""
    st = load().gs_loss_l1_noalloc(C.byref(cam), _f32(color, "color"), _f32(depth, "depth"),
                                   _f32(target_rgb, "target_rgb"), _f32(target_depth, "target_depth"), float(w_color),
                                   float(w_depth), _f32(loss, "loss"), _f32(dL_dcolor, "dL_dcolor"),
                                   _f32(dL_ddepth, "dL_ddepth"), _stream(stream))
    _check(None, st, "gs_loss_l1_noalloc")


def gs_adam_step(ctx, params, grads, m, v, n: int, sh_degree: int, cfg: gs_adam_cfg, step: int, stream=None):
    st = load().gs_adam_step(ctx, _f32(params, "params"), _f32(grads, "grads"), _f32(m, "m"), _f32(v, "v"), int(n),
                             int(sh_degree), C.byref(cfg), int(step), _stream(stream))
    _check(ctx, st, "gs_adam_step")


def gs_bin_tiles(ctx, mean2d, extent, depth, width, height, tile_w, tile_h, keys, ids, ranges, stream=None) -> int:
    n = mean2d.shape[0]
    cap = 0 if keys is None else keys.numel()
    npairs = C.c_int64(0)
    st = load().gs_bin_tiles(ctx, int(n), _f32(mean2d, "mean2d"), _f32(extent, "extent"), _f32(depth, "depth"),
                             int(width), int(height), int(tile_w), int(tile_h), _ptr(keys), _ptr(ids), _ptr(ranges),
                             int(cap), C.byref(npairs), _stream(stream))
    if st == 3:  # capacity: report the size needed
        return -int(npairs.value) - 1
    _check(ctx, st, "gs_bin_tiles")
    return int(npairs.value)


def gs_get_projection(ctx, mean2d=None, cov2d=None, depth=None, rgb=None, opacity=None, tiles=None, stream=None):
    st = load().gs_get_projection(ctx, _f32(mean2d, "mean2d"), _f32(cov2d, "cov2d"), _f32(depth, "depth"),
                                  _f32(rgb, "rgb"), _f32(opacity, "opacity"), _ptr(tiles), _stream(stream))
    _check(ctx, st, "gs_get_projection")


# ---------------------------------------------------------------------------
# batched multi-view entry points: per-view arguments are Python sequences
# ---------------------------------------------------------------------------
def _cams(cams):
    arr = (gs_camera * len(cams))(*cams)
    return arr


def _views(views):
    return (gs_viewmat * len(views))(*views)


def _ptrs(tensors, name, n):
    """Host array of n device pointers (None -> NULL array / entry)."""
    if tensors is None:
        return None
    if len(tensors) != n:
        raise ValueError(f"{name}: expected {n} entries")
    return (C.c_void_p * n)(*[_f32(t, name) for t in tensors])


def gs_render_fwd_batched(ctx, gaussians: gs_gaussians, cams, views, cfg: gs_raster_cfg, color=None, depth=None,
                          alpha=None, stream=None):
    V = len(cams)
    st = load().gs_render_fwd_batched(ctx, C.byref(gaussians), V, _cams(cams), _views(views), C.byref(cfg),
                                      _ptrs(color, "color", V), _ptrs(depth, "depth", V), _ptrs(alpha, "alpha", V),
                                      _stream(stream))
    _check(ctx, st, "gs_render_fwd_batched")


def gs_render_bwd_batched(ctx, gaussians, cams, views, cfg, dL_dcolor, dL_ddepth, dL_dalpha, grads: gs_grads,
                          dL_dpose=None, stream=None):
    V = len(cams)
    st = load().gs_render_bwd_batched(ctx, C.byref(gaussians), V, _cams(cams), _views(views), C.byref(cfg),
                                      _ptrs(dL_dcolor, "dL_dcolor", V), _ptrs(dL_ddepth, "dL_ddepth", V),
                                      _ptrs(dL_dalpha, "dL_dalpha", V), C.byref(grads), _f32(dL_dpose, "dL_dpose"),
                                      _stream(stream))
    _check(ctx, st, "gs_render_bwd_batched")


def gs_render_bwd_adam_batched(ctx, gaussians, cams, views, cfg, dL_dcolor, dL_ddepth, dL_dalpha, params, m, v,
                               adam: gs_adam_cfg, step: int, dL_dpose=None, stream=None):
    V = len(cams)
    st = load().gs_render_bwd_adam_batched(ctx, C.byref(gaussians), V, _cams(cams), _views(views), C.byref(cfg),
                                           _ptrs(dL_dcolor, "dL_dcolor", V), _ptrs(dL_ddepth, "dL_ddepth", V),
                                           _ptrs(dL_dalpha, "dL_dalpha", V), _f32(params, "params"), _f32(m, "m"),
                                           _f32(v, "v"), C.byref(adam), int(step), _f32(dL_dpose, "dL_dpose"),
                                           _stream(stream))
    _check(ctx, st, "gs_render_bwd_adam_batched")


def gs_loss_l1_batched(ctx, cams, color, depth, target_rgb, target_depth, w_color, w_depth, loss, dL_dcolor,
                       dL_ddepth, stream=None):
    V = len(cams)
    st = load().gs_loss_l1_batched(ctx, V, _cams(cams), _ptrs(color, "color", V), _ptrs(depth, "depth", V),
                                   _ptrs(target_rgb, "target_rgb", V), _ptrs(target_depth, "target_depth", V),
                                   float(w_color), float(w_depth), _f32(loss, "loss"),
                                   _ptrs(dL_dcolor, "dL_dcolor", V), _ptrs(dL_ddepth, "dL_ddepth", V),
                                   _stream(stream))
    _check(ctx, st, "gs_loss_l1_batched")


AUTOTUNE_SHAPES = ((16, 16), (8, 32), (32, 8))


def gs_autotune(ctx, gaussians, cams, views, cfg: gs_raster_cfg, reps: int = 5, stream=None) -> list:
    """Picks the fastest tile shape for these views into ``cfg`` (in place);
    returns the milliseconds per pass of each candidate (AUTOTUNE_SHAPES)."""
    ms = (C.c_float * len(AUTOTUNE_SHAPES))()
    st = load().gs_autotune(ctx, C.byref(gaussians), len(cams), _cams(cams), _views(views), C.byref(cfg), int(reps),
                            ms, _stream(stream))
    _check(ctx, st, "gs_autotune")
    return list(ms)


def gs_train_step(ctx, gaussians, cam, view, cfg, target_rgb, target_depth, w_color, w_depth, loss, params, m, v,
                  adam: gs_adam_cfg, step: int, stream=None):
    st = load().gs_train_step(ctx, C.byref(gaussians), C.byref(cam), C.byref(view), C.byref(cfg),
                              _f32(target_rgb, "target_rgb"), _f32(target_depth, "target_depth"), float(w_color),
                              float(w_depth), _f32(loss, "loss"), _f32(params, "params"), _f32(m, "m"), _f32(v, "v"),
                              C.byref(adam), int(step), _stream(stream))
    _check(ctx, st, "gs_train_step")


def gs_train_step_batched(ctx, gaussians, cams, views, cfg, target_rgb, target_depth, w_color, w_depth, loss, params,
                          m, v, adam: gs_adam_cfg, step: int, color=None, depth=None, alpha=None, stream=None):
    V = len(cams)
    st = load().gs_train_step_batched(ctx, C.byref(gaussians), V, _cams(cams), _views(views), C.byref(cfg),
                                      _ptrs(target_rgb, "target_rgb", V), _ptrs(target_depth, "target_depth", V),
                                      float(w_color), float(w_depth), _f32(loss, "loss"), _f32(params, "params"),
                                      _f32(m, "m"), _f32(v, "v"), C.byref(adam), int(step),
                                      _ptrs(color, "color", V), _ptrs(depth, "depth", V), _ptrs(alpha, "alpha", V),
                                      _stream(stream))
    _check(ctx, st, "gs_train_step_batched")


def gs_quadtree_leaves(ctx, rgb, var_thr=0.01, max_size=64, min_size=1, leaves=None, stream=None) -> int:
    """Quadtree leaves of rgb [3, H, W] into ``leaves`` (int32 [cap, 4]);
    returns their number (-needed - 1 if ``leaves`` is too small)."""
    H, W = rgb.shape[1], rgb.shape[2]
    cap = 0 if leaves is None else leaves.shape[0]
    n = C.c_int64(0)
    st = load().gs_quadtree_leaves(ctx, _f32(rgb, "rgb"), int(W), int(H), float(var_thr), int(max_size), int(min_size),
                                   _ptr(leaves), int(cap), C.byref(n), _stream(stream))
    if st == 3:
        return -int(n.value) - 1
    _check(ctx, st, "gs_quadtree_leaves")
    return int(n.value)


def gs_seed_quadtree(ctx, rgb, depth, alpha, alpha_thr, cam: gs_camera, view: gs_viewmat, sh_degree, var_thr,
                     max_size, min_size, means, log_scales, quats, opacity_logits, sh, capacity, stream=None) -> int:
    """Seeds new Gaussians into the given rows; returns how many (-needed - 1
    if more than ``capacity``)."""
    n = C.c_int64(0)
    st = load().gs_seed_quadtree(ctx, _f32(rgb, "rgb"), _f32(depth, "depth"), _f32(alpha, "alpha"), float(alpha_thr),
                                 C.byref(cam), C.byref(view), int(sh_degree), float(var_thr), int(max_size),
                                 int(min_size), _f32(means, "means"), _f32(log_scales, "log_scales"),
                                 _f32(quats, "quats"), _f32(opacity_logits, "opacity_logits"), _f32(sh, "sh"),
                                 int(capacity), C.byref(n), _stream(stream))
    if st == 3:
        return -int(n.value) - 1
    _check(ctx, st, "gs_seed_quadtree")
    return int(n.value)


def gs_tsdf_integrate(ctx, grid: gs_tsdf_grid, depth, cam: gs_camera, view: gs_viewmat, frame: int, min_slot: int = 0,
                      stream=None):
    _check(ctx, load().gs_tsdf_integrate(ctx, C.byref(grid), _f32(depth, "depth"), C.byref(cam), C.byref(view),
                                         int(frame), int(min_slot), _stream(stream)), "gs_tsdf_integrate")


def gs_tsdf_counters(ctx, grid: gs_tsdf_grid, stream=None):
    """(counters [4], status): slots handed out, buckets touched, failed
    inserts, voxels updated; status GS_ERR_CAPACITY (3) when the pool or the
    table is too small."""
    out = (C.c_int64 * 4)()
    st = load().gs_tsdf_counters(ctx, C.byref(grid), out, _stream(stream))
    if st not in (GS_OK, 3):
        _check(ctx, st, "gs_tsdf_counters")
    return [int(v) for v in out], st


def gs_tsdf_rehash(ctx, src: gs_tsdf_grid, dst: gs_tsdf_grid, stream=None):
    _check(ctx, load().gs_tsdf_rehash(ctx, C.byref(src), C.byref(dst), _stream(stream)), "gs_tsdf_rehash")


def gs_tsdf_query(ctx, grid: gs_tsdf_grid, points, tsdf=None, weight=None, stream=None):
    _check(ctx, load().gs_tsdf_query(ctx, C.byref(grid), _f32(points, "points"), int(points.shape[0]),
                                     _f32(tsdf, "tsdf"), _f32(weight, "weight"), _stream(stream)), "gs_tsdf_query")


def gs_seed_tsdf(ctx, rgb, depth, grid: gs_tsdf_grid, cam: gs_camera, view: gs_viewmat, sh_degree, var_thr, max_size,
                 min_size, means, log_scales, quats, opacity_logits, sh, capacity, stream=None) -> int:
    """Seeds new Gaussians (voxel-weight novelty) into the given rows; returns
    how many (-needed - 1 if more than ``capacity``)."""
    n = C.c_int64(0)
    st = load().gs_seed_tsdf(ctx, _f32(rgb, "rgb"), _f32(depth, "depth"), C.byref(grid), C.byref(cam), C.byref(view),
                             int(sh_degree), float(var_thr), int(max_size), int(min_size), _f32(means, "means"),
                             _f32(log_scales, "log_scales"), _f32(quats, "quats"),
                             _f32(opacity_logits, "opacity_logits"), _f32(sh, "sh"), int(capacity), C.byref(n),
                             _stream(stream))
    if st == 3:
        return -int(n.value) - 1
    _check(ctx, st, "gs_seed_tsdf")
    return int(n.value)


def gs_count_nonfinite(ctx, x, stream=None) -> int:
    """Number of NaN / +-Inf values in the float32 device tensor x."""
    n = C.c_int64(0)
    st = load().gs_count_nonfinite(ctx, _f32(x, "x"), int(x.numel()), C.byref(n), _stream(stream))
    if st not in (GS_OK, 4):
        _check(ctx, st, "gs_count_nonfinite")
    return int(n.value)


def gs_ctx_inject_alloc_failure(ctx, after: int = 1):
    _check(ctx, load().gs_ctx_inject_alloc_failure(ctx, int(after)), "gs_ctx_inject_alloc_failure")


def gs_bounds_checked() -> bool:
    """True when the loaded library is the bounds-checked build."""
    return bool(load().gs_bounds_checked())


def gs_ctx_inject_bounds_fault(ctx):
    _check(ctx, load().gs_ctx_inject_bounds_fault(ctx), "gs_ctx_inject_bounds_fault")


def gs_get_tile_ranges(ctx, ranges, stream=None):
    """ranges: int32 CUDA tensor [n_tiles, 2] receiving [first, last + 1) per tile."""
    _check(ctx, load().gs_get_tile_ranges(ctx, _ptr(ranges), int(ranges.shape[0]), _stream(stream)),
           "gs_get_tile_ranges")


def gs_get_tile_order(ctx, order, stream=None):
    """order: int32 CUDA tensor [n_tiles] receiving the raster visit order."""
    _check(ctx, load().gs_get_tile_order(ctx, _ptr(order), int(order.shape[0]), _stream(stream)),
           "gs_get_tile_order")


def gs_state_token(ctx) -> int:
    """Token of the forward state the context holds (0 = none)."""
    tok = C.c_uint64(0)
    _check(ctx, load().gs_state_token(ctx, C.byref(tok)), "gs_state_token")
    return int(tok.value)


def gs_measure_alu_peaks(device: int = 0, iters: int = 50000) -> dict:
    out = gs_alu_peaks()
    _check(None, load().gs_measure_alu_peaks(int(device), int(iters), C.byref(out)), "gs_measure_alu_peaks")
    return {name: getattr(out, name) for name, _ in gs_alu_peaks._fields_}
