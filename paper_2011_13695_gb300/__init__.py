"""GB300-native dual-polarisation coherent receiver (sm_103a CUDA behind a C ABI).

``rx`` is the ctypes binding of ``librx.so`` (declared in ``include/rx.h``);
``receiver`` wraps it for torch device buffers; ``build`` compiles the
library with nvcc. Nothing here computes any part of the receiver in Python.
"""

from . import rx  # noqa: F401

__all__ = ["rx"]
