"""GB300-native AIMx: the accelerated surface-integral-equation matvec, solve and sweep.

The compute path is the CUDA library ``libaimx.so`` (sources in ``csrc/``, C ABI in
``include/aimx.h``); ``aimx`` is its thin ctypes binding.
"""

from .aimx import (AimxError, Batch, Context, Gnn, Port, EFIE, PMCHWT, CFIE, F32, F64, PRECOND_DIAG, PRECOND_NONE,  # noqa: F401
                   PRECOND_BLOCK, PRECOND_LEARNED, load, wait_timeouts)
