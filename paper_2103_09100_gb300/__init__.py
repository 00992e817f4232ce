"""GB300 explicit solver for elasto-dynamics on 2:1-balanced octree meshes.

The central-difference time step of the octree SBFEM method (Zhang et al.,
arXiv 2103.09100): element-by-element internal force from a few precomputed
master-cell stiffness matrices, then the lumped-mass update, run as
hand-written sm_103a CUDA kernels behind the C ABI of ``include/sbx.h``.

* ``_lib``     -- ctypes binding of the C ABI (same names)
* ``build``    -- nvcc build of ``_build/libsbx.so``
* ``patterns`` -- host set-up: master-cell classification and SBFEM pattern
                  matrices (Sec. 2, 3.2, 3.3)
* ``solver``   -- ``Solver``: one-call set-up of a mesh on the GPU
"""
from . import _lib  # noqa: F401
from .solver import Solver  # noqa: F401
