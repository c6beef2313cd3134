"""GB300 mixed-FEM skinning pose solver: CUDA library (csrc/, include/mfem.h)
and its thin ctypes binding (mfem.py)."""
from . import build  # noqa: F401

__all__ = ["build", "mfem"]
