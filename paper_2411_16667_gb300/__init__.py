"""GB300-native exact multi-objective shortest-path search (OPMOS method).

The compute path is the CUDA library ``libopmos.so`` (C ABI in
``include/opmos.h``); ``opmos`` is its ctypes binding. There is no CPU
fallback: every call fails loudly if the library or a CUDA device is missing.
"""
from .build import build  # noqa: F401
