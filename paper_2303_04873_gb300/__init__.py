"""GB300 (sm_103a) evaluator of MOREA's objectives and fold constraint.

The work happens in ``libmorea.so`` (hand-written CUDA kernels behind the C
ABI declared in ``include/morea.h``); ``morea`` is its ctypes binding and
``build`` compiles it in-tree.
"""

__all__ = ["build", "morea"]
