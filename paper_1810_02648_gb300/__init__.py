"""GB300-native (sm_103a) Gauss-Newton hot path of LiveCap (arXiv 1810.02648).

The compute lives in the CUDA library ``_lib/liblivecap.so`` (C ABI declared
in ``include/livecap.h``); ``livecap`` is its ctypes binding.  There is no
CPU fallback: without the built library and a CUDA device every call fails.
"""
from .livecap import MLP, Batch, Context, LivecapError, load  # noqa: F401
