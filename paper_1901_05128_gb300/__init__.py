"""GB300-native convolution-quadrature history sums and two-state fractional
Fokker-Planck schemes (arXiv 1901.05128).

The compute path is the CUDA library ``_build/libfastcq.so`` (sources in
``csrc/``, C ABI in ``include/fastcq.h``); ``fastcq`` is its ctypes binding.
Build it with ``paper_1901_05128_gb300.build.build()``.
"""
from .build import build  # noqa: F401


def load():
    """Import and return the binding module (raises ImportError if the library is not built)."""
    from . import fastcq
    return fastcq
