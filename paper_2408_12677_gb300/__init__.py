"""GB300 (sm_103a) differentiable 3D Gaussian splatting hot path of GSFusion
(arXiv 2408.12677): tile rasterizer forward/backward and the Adam update,
behind the C ABI of ``include/gsplat.h`` (libgsplat.so, built in-tree by
``paper_2408_12677_gb300.build``).

``abi``        ctypes binding, same names as the C entry points.
``torch_api``  flat-buffer Gaussian model, single-view and batched trainers,
               autograd Function, trainer checkpoints.
``streaming``  the per-frame loop: TSDF fusion, seeding, keyframes, batched
               iterations, global optimisation, checkpoints of the loop.
``tsdf``       buffers of the TSDF grid (sizing only; the fusion runs in the
               library).
``checkpoint`` the map checkpoint file format.
"""
from . import abi  # noqa: F401

__all__ = ["abi"]
