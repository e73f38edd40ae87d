"""GB300-native Maxwell-Liouville-von Neumann solver (Riesch & Jirauschek,
arXiv:1710.09799): Strang splitting in the SU(N) adjoint representation with
the diagonalised interaction exponential, fused with 1D FDTD, on sm_103a.

The compute path is libmln.so (include/mln.h); `mln` is its ctypes binding.
"""
from . import mln
from .mln import Params, Solver, MLNError

__all__ = ["mln", "Params", "Solver", "MLNError", "build"]


def build(force: bool = False) -> str:
    from ._nvcc_build import build as _build
    return _build(force=force)
