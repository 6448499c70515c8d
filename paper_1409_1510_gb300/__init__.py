"""GB300 (sm_103a) multi-right-hand-side even-odd HISQ Dslash and CG solvers.

The computation lives in the CUDA library ``libhisq_gb300.so`` (C ABI in ``include/hisq.h``);
``paper_1409_1510_gb300.hisq`` is its ctypes binding with the same function names.
"""
from . import accounting  # noqa: F401
