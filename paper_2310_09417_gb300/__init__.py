"""GB300-native randomized column interpolative decomposition (arXiv:2310.09417).

The compute path lives in the CUDA library built from ``csrc/`` (C-ABI declared
in ``include/randid.h``); :mod:`paper_2310_09417_gb300.binding` marshals
arguments to it.  Importing this package does not load the library; the first
call into the binding does, and fails loudly if it has not been built.
"""
