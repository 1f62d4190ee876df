"""FP64 CPU oracle for the differentiable tile-based 3D Gaussian splatting
rasterizer and its Adam update (GSFusion, Sec. III-A.2 and III-B.3).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain definition that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_2408_12677_gb300``) never imports it and shares no
code with it; both sides only share the seeded input generators in ``synth/``.
Those hold none of the rasterizer's arithmetic, but ``synth.quadtree`` seeds
the synthetic Gaussian sets with the paper's quadtree and Eq. 10 (input
plumbing, on the host); ``oracle.quadtree`` is a separate implementation of
the same seeding, written independently and cross-checked against it.

Modules
-------
``sh``       real spherical-harmonic basis up to degree 3, built from the
             Legendre-polynomial definition (pinned against scipy's complex
             spherical harmonics and by quadrature orthonormality).
``render``   projection (Eq. 2-5), per-pixel front-to-back compositing with no
             tiling (Eq. 11), the L1 loss (Eq. 12) and gradients by PyTorch
             autograd in float64.
``adam``     the Adam update with per-group learning rates (float64).
``binning``  the integer tile-binning rule: (tile, depth) keys, stable sort,
             per-tile ranges (numpy, bit-exact).
``quadtree`` the per-frame seeding: contrast quadtree over the RGB frame and
             the back-projection of its leaf centres (Eq. 10).
``tsdf``     the TSDF fusion (Eq. 6-9) over 8^3-voxel blocks and the
             voxel-weight novelty check of the seeding.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py`` to
something other than itself (closed forms, Monte Carlo, finite differences,
library routines, brute force).  No function is "parity unpinned".
"""
from . import adam, binning, quadtree, render, sh, tsdf  # noqa: F401
