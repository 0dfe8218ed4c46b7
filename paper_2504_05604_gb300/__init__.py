"""GB300-native SIMP + Optimality Criteria hot path (arXiv 2504.05604).

The compute lives in the CUDA library ``libto3d.so`` (sources in ``csrc/``,
interface in ``include/to3d.h``); ``binding`` is its ctypes binding.
"""
from .binding import (  # noqa: F401
    Batch, Context, To3dError, default_params, load, exported_symbols, conv3d_forward,
    conv3d_backward, sensitivity_noalloc,
    F64, BF16_DC, BF16X2_DC, FP16_DC, FP16X2_DC, JACOBI, CNN_FCG, LMG, FILTER_SENS, FILTER_DENS,
)
