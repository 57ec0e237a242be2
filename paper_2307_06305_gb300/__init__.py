"""GB300-native DA-CSR sparse matrix library (Saak & Schulze, arXiv 2307.06305).

The compute path is the CUDA library ``_lib/libdamn.so`` built from ``csrc/``
for sm_103a (C ABI in ``include/damn.h``); ``damn`` is its thin Python
binding.  This ``__init__`` imports nothing so that the package can be
inspected without a GPU; use ``from paper_2307_06305_gb300 import damn``.
"""
