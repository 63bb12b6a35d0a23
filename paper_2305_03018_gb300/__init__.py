"""GB300 (sm_103a) library for exact grey-value dilation and erosion by
umbra / polynomial convolution (arxiv 2305.03018).

The computation lives in the CUDA library ``_lib/libmorph_gb300.so`` (C ABI
in ``include/morph.h``); :mod:`.morph` is its ctypes binding and
:mod:`.autograd` the PyTorch layer.  :mod:`.workloads` draws seeded inputs.
"""
from .morph import (Context, MorphError, get_context, load_library)  # noqa: F401

__all__ = ["Context", "MorphError", "get_context", "load_library"]
