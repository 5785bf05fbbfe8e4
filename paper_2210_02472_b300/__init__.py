"""libfsi: B300-native hot path of a fourth-order forward symplectic N-body integrator.

The compute path lives in the CUDA shared library built from ``csrc/``; the Python
module ``paper_2210_02472_b300.fsi`` is a thin ctypes binding over its C ABI.
Importing this package loads nothing; importing ``fsi`` loads the library and fails
loudly if it is missing.
"""
__all__ = ["inputs"]
