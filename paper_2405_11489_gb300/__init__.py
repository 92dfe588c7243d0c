"""GB300-native PonD double-distribution BGK step (arXiv 2405.11489).

The compute path is the C-ABI library ``libpond`` (hand-written sm_103a CUDA kernels,
``csrc/``); ``pond.py`` is its thin ctypes binding.  Importing this package does not
load the library: ``from paper_2405_11489_gb300 import pond`` does, and fails loudly
if the CUDA build is missing.
"""
__all__ = ["pond", "workloads"]
