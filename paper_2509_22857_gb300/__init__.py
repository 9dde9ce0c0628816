"""GB300-native leveled RNS-CKKS inference of quadratic-activation CNNs.

The compute path is the CUDA library ``_build/libfhecnn.so`` (sources in
``csrc/``, C ABI in ``include/fhecnn.h``); ``_lib`` is its thin ctypes
binding and ``model`` lowers a network description into the library's
program format on the host (batch-norm folding, weight redistribution, slot
layouts, diagonals, rescale placement).
"""
from . import _lib  # noqa: F401
from ._lib import FheError  # noqa: F401
