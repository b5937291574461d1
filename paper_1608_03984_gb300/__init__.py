"""GB300-native explicit finite-difference wave solver (arXiv 1608.03984 hot path).

The compute path is libfdwave.so (CUDA, sm_103a) behind the C ABI of
include/fdwave.h; :mod:`.fdwave` is its Python binding and :mod:`.synth`
draws the seeded synthetic workloads. Importing the package loads nothing.
"""
__all__ = ["fdwave", "synth", "build"]
