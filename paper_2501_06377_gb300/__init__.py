"""GB300 (sm_103a) implementation of the HipFT surface-flux-transport step.

The compute path is libsft.so (hand-written CUDA kernels behind the C-ABI
of include/sft.h); ``sft`` is its thin ctypes binding.  Build the library
with ``paper_2501_06377_gb300.build.build()``.
"""
from .sft import (AssimParams, FlowParams, Grid, SFTError, header_functions,  # noqa: F401
                  load, LIB_PATH)

__all__ = ["AssimParams", "FlowParams", "Grid", "SFTError", "header_functions", "load", "LIB_PATH"]
