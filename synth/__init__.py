"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package only *generates inputs*: camera intrinsics and poses, Gaussian
parameter sets and target RGB-D frames.  It holds none of the rasterizer's
arithmetic (projection, compositing, gradients, optimiser); both the FP64
oracle (``oracle/``) and the CUDA path consume what it produces.  It does
implement the paper's quadtree seeding (Eq. 10) to build the Gaussian sets
from its frames: that is method arithmetic used as input plumbing, and the
oracle and the GPU seeding kernels each have their own implementation of it.

Contents
--------
``scene``     a procedural room (floor, ceiling, four walls, 20 boxes) with a
              multi-octave value-noise texture, ray cast on the CPU into an
              RGB-D frame (stand-in for the paper's Replica / ScanNet++ frames,
              which are not available here).
``quadtree``  the paper's contrast quadtree seeding (Sec. III-B.2, Eq. 10):
              split cells while their RGB variance exceeds a threshold, one
              Gaussian per leaf at the back-projected leaf centre.
``workloads`` the five workload recipes (tiny random scene, single view,
              scale stress, uneven multi-view batch, streaming trajectory).
"""
from . import scene, quadtree, workloads  # noqa: F401
