"""GB300-native MLS-MPM substep library (arXiv 2502.18437, CRESSim-MPM hot path).

The compute path is hand-written CUDA for sm_103a behind a C ABI
(``include/mpm.h``); ``paper_2502_18437_gb300.mpm`` is its thin Python binding.
Importing this package loads nothing; the shared library is loaded on first use.
"""
__all__ = ["mpm", "workloads"]
