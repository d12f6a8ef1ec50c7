"""GB300 space-time boundary element library for the 3D heat equation.

Assembly of the block lower-triangular Toeplitz matrices V_h, K_h of the
semi-analytic space-time Galerkin BEM (piecewise-constant basis, uniform
steps), the block-Toeplitz matrix-vector product and the forward-substitution
Dirichlet solve, as hand-written sm_103a CUDA kernels behind the C ABI of
include/stbem.h.  ``capi`` is the ctypes binding of that ABI; ``pipeline``
chains its calls for a whole Dirichlet problem.
"""
from . import capi  # noqa: F401
from .capi import (STB_PREC_FP64, STB_PREC_MIXED, STB_STORE_F32, STB_STORE_F64,  # noqa: F401
                   Mesh, StbError, stb_default_params, stb_launch_count)
