"""FP64 CPU oracle for the LDSolver coarse-grid finite-volume step.

TEST INFRASTRUCTURE ONLY. Nothing in the product path (the CUDA library and its
Python binding) may import, call or link anything in this package; only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference arm of
``bench.py`` use it.

The oracle is a plain, slow, obviously-correct restatement of the method in
numpy float64. It shares no code with the GPU path. Each function cites the
section or equation of the paper (Learnable-Differentiable Finite Volume Solver
for Accelerated Simulation of Flows, KDD'25) that it follows.

Every function here is pinned by tests under ``tests/`` to something other than
itself (closed forms, exact discrete invariants, a dense direct solve, brute
force). Functions without such a pin are marked "parity unpinned" in their
docstring; at present that is only the training outcome, which lives outside
this package.
"""

from .fv import *  # noqa: F401,F403
from .fno import FNOParams, fno_forward, fno_vjp, spectral_conv, spectral_conv_vjp  # noqa: F401
from .scalar import rk4_step_scalar, rollout_scalar, scalar_tendency  # noqa: F401
