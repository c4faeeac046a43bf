"""GB300 (sm_103a) graph-coloured parallel p-bit annealer (arXiv 2510.23419).

The computation lives in the CUDA library ``libpbit.so`` behind the C ABI of
``include/pbit.h``; ``native`` is its thin Python binding.
"""
from . import native  # noqa: F401
from .native import *  # noqa: F401,F403
