"""GB300-native density peaks clustering (PECANN): the data-parallel path as
hand-written sm_103a CUDA behind a C ABI (include/pecann.h).

Modules:
  pecann  -- Python binding of the C ABI (same names as the entry points)
  build   -- in-tree compilation of libpecann.so with nvcc
  synth   -- seeded synthetic inputs (shared by tests and the benchmark)
"""
__all__ = ["pecann", "build", "synth"]
