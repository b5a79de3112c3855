"""GB300 (sm_103a) multi-time-step SPH solid relaxation (arXiv 2309.04010).

The compute path is the CUDA library libmtssph.so (C ABI in include/mtssph.h);
``mtssph`` is its ctypes binding.
"""
from . import mtssph  # noqa: F401
from .mtssph import Body, Context, body_from_case  # noqa: F401

__all__ = ["mtssph", "Body", "Context", "body_from_case"]
