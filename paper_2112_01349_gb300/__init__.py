"""GB300-native bundle adjustment: the LM hot path of MegBA (arXiv 2112.01349).

The computation lives in ``_build/libmba.so`` (hand-written CUDA for sm_103a
behind the C ABI of include/mba.h); ``mba`` is its ctypes binding.
"""
from . import mba  # noqa: F401
from .mba import Problem, MbaError  # noqa: F401
