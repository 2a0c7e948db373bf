"""CGKS-5 CPU oracle (test infrastructure only).

Plain FP64 C implementation of the scheme, loaded through ctypes.  Only the
tests, the smoke check and the CPU-baseline leg of the benchmark may import
this package; the CUDA library never does.
"""
from .oracle import Oracle, build_oracle, lib  # noqa: F401
