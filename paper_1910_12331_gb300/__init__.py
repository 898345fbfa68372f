"""GB300-native Gauss-Newton CP decomposition (hot path).

The compute lives in ``libcpgn.so`` (hand-written CUDA for sm_103a behind a
C ABI declared in ``include/cpgn.h``); ``api`` is a thin ctypes binding with
the same call names.  Importing this package does not load the library;
the first call does, and raises if the library is missing.  There is no CPU
fallback.
"""
from . import datagen  # noqa: F401

__all__ = ["datagen"]
