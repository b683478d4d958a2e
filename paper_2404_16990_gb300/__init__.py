"""GB300-native 2D Ising checkerboard Metropolis simulator.

The compute path is the CUDA library ``libising.so`` (sm_103a) behind the C
ABI declared in ``include/ising.h``; ``paper_2404_16990_gb300.ising`` is the
thin ctypes binding with the same names.  ``workloads`` holds the seeded
synthetic inputs.
"""
__all__ = ["ising", "workloads"]
