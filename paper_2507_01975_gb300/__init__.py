"""GB300-native LDSolver coarse-grid FV step.

The compute path is the CUDA library ``libldfv.so`` built from ``csrc/`` for
sm_103a; ``paper_2507_01975_gb300.fd`` is a thin ctypes binding over its C ABI
(``include/fd.h``). Importing the package loads nothing; the library is loaded
on first use and a missing library is an error, never a fallback.
"""

__all__ = ["fd", "inputs"]
