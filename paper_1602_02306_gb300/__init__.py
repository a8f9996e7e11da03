"""GB300-native preconditioned Lanczos eigenvalue counts (Vecharynski & Yang).

``evc``     -- ctypes binding of the C-ABI library ``libevc.so`` (CUDA, sm_103a).
``inputs``  -- seeded synthetic problem generators.
``build``   -- in-tree nvcc build of ``libevc.so``.
"""
__all__ = ["evc", "inputs", "build"]
