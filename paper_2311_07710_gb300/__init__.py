"""GB300 (sm_103a) restarted accelerated PDHG for convex QP.

The solver lives in the CUDA library libpdqp.so (C ABI in include/pdqp.h);
`pdqp` is its thin ctypes binding and `build` compiles it in-tree.
"""
from . import build  # noqa: F401
