"""Single-GPU (sm_103a) spaND preconditioner with second-order sparsification.

The compute path is the C-ABI library ``libspand.so`` (CUDA kernels and C++
host code under ``csrc/``, interface in ``include/spand.h``).  The Python
module ``spand`` only marshals arguments to it; importing it fails loudly when
the library has not been built.
"""

FIRST_ORDER = 0
SECOND_ORDER_FULL = 1
SECOND_ORDER_SUPERFINE = 2

__all__ = ["FIRST_ORDER", "SECOND_ORDER_FULL", "SECOND_ORDER_SUPERFINE"]
