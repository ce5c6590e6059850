"""Warp-collective library for GB300 (sm_103a).

The compute path lives in ``libcox.so`` (CUDA kernels behind the C-ABI of
``include/cox.h``); ``paper_2112_10034_gb300.cox`` is its thin ctypes binding.
Importing this package loads nothing: ``inputs`` (seeded workload
generators) is usable without a GPU.
"""
