"""GB300-native DEM contact pipeline (arXiv 2311.04648, Chrono DEM-Engine).

The compute path is the C-ABI library ``libdem_gb300.so`` built from ``csrc/`` (hand-written
CUDA for sm_103a); ``dem`` is its thin ctypes binding and ``workloads`` holds the seeded
synthetic scene generators.  Importing this package loads nothing; ``dem.load()`` loads
the library and fails loudly if it is missing.
"""
__all__ = ["dem", "workloads"]
