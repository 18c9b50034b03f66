"""GB300-native multigrid Poisson solver (HONEI paper, arXiv 0904.4152): Q1 FEM on the unit square,
9-band operator, damped-Jacobi V cycles and mixed-precision defect correction in hand-written
sm_103a CUDA behind a C ABI (``include/hn.h``).

Submodules: ``hn`` (ctypes binding of the C ABI, loads ``libhn.so``), ``build`` (nvcc build of the
library), ``inputs`` (seeded synthetic problem generators).  Importing the package loads nothing.
"""
__all__ = ["hn", "build", "inputs"]
