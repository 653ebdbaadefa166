"""GB300 free-space Spectral Ewald summation of stokeslet, stresslet and rotlet sums.

The compute path is the CUDA library ``libse.so`` (C ABI in ``include/se.h``);
``se`` is its ctypes binding.  Build with ``paper_1607_04808_gb300._build.build()``.
"""
from .se import (KERNELS, Batch, Plan, SEError, SEFunction, choose_params, choose_params_points, se_sum,  # noqa: F401
                 measure_peaks, set_precompute_cache, version)
