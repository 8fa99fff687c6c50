"""GB300-native Chebyshev-filtered plane-wave Hamiltonian application (arxiv 2604.11139).

The compute path lives in the CUDA library built from csrc/ (C ABI: include/pw.h);
``pwlib`` is its ctypes binding.  ``workloads`` draws the seeded synthetic inputs.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "pwlib", "build"]
