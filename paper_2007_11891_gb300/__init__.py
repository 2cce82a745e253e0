"""GB300-native statically condensed HDG operator and solver (arXiv:2007.11891).

The compute path is the in-tree CUDA library ``lib/libhdg_gb300.so``
(sm_103a) behind the C ABI of ``include/hdg.h``; this package only marshals
arguments (``_capi``) and wraps torch tensors (``hdg``).
"""
from .hdg import HDG, HDGLowDim, HDGSolve, measure_fma_peak  # noqa: F401
