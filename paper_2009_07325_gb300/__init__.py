"""GB300-native IMM: RR-set sampling (IC, LT) and greedy max coverage in CUDA.

The library is ``libgim.so`` (C ABI in include/gim.h); ``binding`` is its
ctypes binding and ``inputs`` holds the seeded synthetic graph generators.
"""
from .binding import GIM_IC, GIM_LT, Context, GimError, load_library  # noqa: F401
