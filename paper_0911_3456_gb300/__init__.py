"""GB300 (sm_103a) filter-bank correlation: the data-parallel hot path of the
vision case study of "PyCUDA and PyOpenCL: A Scripting-Based Approach to GPU
Run-Time Code Generation" (Sec. 6.2), rebuilt around run-time-generated,
auto-tuned CUDA kernels behind a C ABI (include/fbcorr.h); plus the exact
nearest-neighbour search of its natural-scene case study (Sec. 6.4, NNPlan).

Importing this package does not load the CUDA library; the first plan does.
"""
__all__ = ["Plan", "BatchPlan", "NNPlan", "FBCorr", "fbcorr", "get_plan"]


def __getattr__(name):
    if name in __all__:
        from . import api as _m
        return getattr(_m, name)
    raise AttributeError(name)
