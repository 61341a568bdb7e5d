"""GB300-native parallel bounding for the permutation flow-shop branch-and-bound.

The compute path lives in the CUDA library built from ``csrc/`` (C-ABI declared
in ``include/fsp.h``); ``fsp`` is its thin Python binding and ``inputs`` the
seeded synthetic workloads.  Import ``paper_1206_4973_gb300.fsp`` explicitly:
this package init loads nothing.
"""
