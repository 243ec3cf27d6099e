"""GB300-native DGSEM for the compressible Navier-Stokes equations (the method of
GALAEXI, arXiv 2404.12703): hand-written sm_103a CUDA kernels behind a C ABI
(``include/dg.h``), a thin ctypes binding (``dg``), and seeded synthetic
workloads (``workloads``).

Importing the package does not load the CUDA library; ``dg.load()`` does, and
fails loudly if it is missing.
"""
__all__ = ["dg", "workloads", "build"]
