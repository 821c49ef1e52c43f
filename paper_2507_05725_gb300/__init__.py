"""GB300 (sm_103a) FTH-MS open-arc hot path: CUDA library libfthms.so + its C ABI binding.

Layout:
  csrc/      CUDA kernels (kernels.cu, bessel.cuh), host planner (plan.cpp), C ABI (api.cu)
  build.py   nvcc build of lib/libfthms.so (in-tree)
  fthms.py   ctypes binding with the C names (argument marshalling only)
"""
__all__ = ["build", "fthms"]


def build(**kw):
    from .build import build as _b
    return _b(**kw)
