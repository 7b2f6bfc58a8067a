"""B300 (sm_103a) distillation solver for the domain-decomposition subtraction estimator of
quark-line disconnected correlators.

The compute path is the CUDA library liblqcd.so (C ABI in include/lqcd.h); ``lqcd`` is its thin
ctypes binding with the same entry-point names.  Importing the package loads the library and
fails loudly if it has not been built (``python -m paper_2609_37049_b300.build``).
"""
from . import lqcd  # noqa: F401  (loads liblqcd.so)
from .lqcd import Context, Stats, default_params, LqcdError  # noqa: F401
from . import autotune  # noqa: F401

__all__ = ["lqcd", "autotune", "Context", "Stats", "default_params", "LqcdError"]
