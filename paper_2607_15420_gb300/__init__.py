"""GB300 (sm_103a) library for the scenario-based absorber design problem (problem (10)).

The hot path -- the fused evaluation of residuals, Jacobian and Lagrangian Hessian, the
block-LU / Schur-on-diameter KKT factorization and solve, FP64 refinement and the
interior-point iteration -- runs in the CUDA library libabsorber.so (C ABI declared in
include/absorber.h).  `binding` is its ctypes wrapper; `build` compiles it in-tree.
"""
from . import build  # noqa: F401


def load():
    """The ctypes binding module, with the library loaded (raises if not built)."""
    from . import binding
    binding.lib()
    return binding
