"""GB300-native FFT stencil solver (arXiv 2105.06676: StencilFFT-P / StencilFFT-A).

The compute path is libstencilfft.so (hand-written sm_103a CUDA behind a C
ABI, include/stencilfft.h); this package is its thin Python binding.
"""
from . import workloads  # noqa: F401  (seeded inputs; no arithmetic of the method)

__all__ = ["StencilPlan", "VectorStencilPlan", "BatchExecutor", "StencilServer", "solve", "max_axis", "workspace_bytes", "StencilError",
           "workloads"]


def __getattr__(name):
    if name in ("StencilPlan", "VectorStencilPlan", "BatchExecutor", "StencilServer", "solve",
                "max_axis", "workspace_bytes"):
        from . import api
        return getattr(api, name)
    if name == "StencilError":
        from ._capi import StencilError
        return StencilError
    raise AttributeError(name)
