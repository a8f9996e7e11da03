"""Plain FP64 CPU oracle of the preconditioned Lanczos eigenvalue-count estimator.

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg use this package. It shares no code with the
CUDA library and never imports it.
"""
from .oracle import *  # noqa: F401,F403
