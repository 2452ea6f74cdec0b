"""GB300-native QUAPI tensor-propagator library (Python side).

The compute path lives in ``libquapi.so`` (hand-written sm_103a CUDA kernels
behind a C ABI, declared in ``include/quapi.h``).  ``quapi`` is the thin
ctypes binding with the same entry-point names; ``workloads`` holds the seeded
synthetic problem inputs.  Importing this package does not load the library;
the first call into ``quapi`` does, and fails loudly if it is missing.
"""

__all__ = ["quapi", "workloads"]
