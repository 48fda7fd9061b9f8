"""GB300 (sm_103a) Gauss-Newton-Krylov diffeomorphic image registration.

A from-scratch implementation of the hot path of the method of Brunn et al.,
arXiv 2008.12820 (CLAIRE): reduced gradient and Gauss-Newton Hessian matvec
inside PCG, built from semi-Lagrangian transport (RK2 characteristics,
periodic cubic Lagrange interpolation) and spectral operators, behind the C
ABI of ``include/claire.h``.  ``claire`` is the Python binding; ``synth`` makes
the seeded synthetic inputs; ``build`` compiles the CUDA library in-tree.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "claire", "build"]
