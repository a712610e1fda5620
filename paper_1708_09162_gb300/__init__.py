"""GB300 (sm_103a) isogeometric single-layer BEM with interpolation FMM.

The compute path is libibem (CUDA, C ABI in include/ibem.h); ``ibem`` is its
ctypes binding.  Build the library with ``paper_1708_09162_gb300.build.build()``.
"""
