"""GB300-native banded Smith-Waterman seed extension (BSW).

The library (libbsw.so, built from csrc/ for sm_103a) exposes the C ABI in
include/bsw.h; ``bsw`` is its Python binding and ``workload`` draws the
seeded synthetic inputs.
"""
__all__ = ["bsw", "build", "workload"]
