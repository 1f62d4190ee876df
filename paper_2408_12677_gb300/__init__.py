"""GB300 (sm_103a) differentiable 3D Gaussian splatting hot path of GSFusion
(arXiv 2408.12677): tile rasterizer forward/backward and the Adam update,
behind the C ABI of ``include/gsplat.h`` (libgsplat.so, built in-tree by
``paper_2408_12677_gb300.build``).

``abi``        ctypes binding, same names as the C entry points.
``torch_api``  flat-buffer Gaussian model, one-iteration trainer, autograd
               Function.
"""
from . import abi  # noqa: F401

__all__ = ["abi"]
