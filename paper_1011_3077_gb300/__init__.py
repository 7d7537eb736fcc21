"""GB300-native inverse-free spectral divide-and-conquer eigensolver.

The compute path lives in the C-ABI library built from ``csrc/`` (see
``include/eigdc.h``); :mod:`paper_1011_3077_gb300.eigdc` is the thin ctypes
binding with the same entry-point names.  :mod:`workloads` builds the seeded
synthetic inputs.
"""
