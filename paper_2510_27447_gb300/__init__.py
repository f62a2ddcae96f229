"""GB300 (sm_103a) library for the partitioned bidomain time step with
spectral deferred correction.

The compute path lives in ``csrc/`` (CUDA C++ behind a C ABI declared in
``include/bd.h``); ``binding`` loads the shared library with ctypes.  Importing
this package does not load the library; ``workloads`` holds the seeded
synthetic inputs.
"""
__all__ = ["workloads"]
