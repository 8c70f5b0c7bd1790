"""GB300-native memory-efficient Strassen-Winograd matrix multiplication.

The computation lives in the C-ABI library libswmm.so (include/swmm.h);
`swmm` is its thin ctypes binding.  Build the library with
`paper_0707_2347_gb300.build.build()`.
"""
from . import swmm  # noqa: F401
from .swmm import Handle, Opts, SwmmError  # noqa: F401
