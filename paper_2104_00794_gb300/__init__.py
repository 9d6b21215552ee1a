"""GB300-native probed (randomized-trace) FWI gradient, arXiv 2104.00794.

Submodules:
  native     ctypes binding of the C-ABI library ``libtprobe.so`` (CUDA, sm_103a)
  api        torch-facing helpers (workspace allocation, batched calls)
  workloads  seeded synthetic inputs (models, geometry, wavelet)
"""
__all__ = ["native", "api", "workloads"]
