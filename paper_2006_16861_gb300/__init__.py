"""GB300-native time-domain Helmholtz preconditioner (Stolk, arXiv 2006.16861).

Modules:
  htd        ctypes binding of libhtd.so (the C ABI in include/htd.h)
  workloads  seeded synthetic problem inputs (no method arithmetic)
  _native    in-tree build of libhtd.so for sm_103a

Importing the package loads nothing native; ``htd.load()`` does.
"""
__all__ = ["htd", "workloads"]
