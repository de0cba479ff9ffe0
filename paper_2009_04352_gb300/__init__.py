"""GB300-native LBM-LES channel solver with the wall-function bounce boundary
(Han, Ooka & Kikumoto, arXiv 2009.04352).

The compute path is the CUDA C-ABI library built from ``csrc/`` (declared in
``include/lbm.h``); ``lbm`` is its thin ctypes binding and ``workload`` the
seeded synthetic channel recipes. Importing the package does not load the
library; the first use of ``lbm`` does, and fails loudly if it is not built.
"""
__all__ = ["lbm", "workload", "build"]
