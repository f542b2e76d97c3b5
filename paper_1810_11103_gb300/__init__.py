"""GB300-native WENOIU free-stream-preserving Euler right-hand side (arXiv:1810.11103).

The compute path lives in the CUDA library ``libfsp.so`` (C ABI, ``include/fsp.h``);
``paper_1810_11103_gb300.fsp`` is its thin Python binding.  Importing this package does
not load the library; ``inputs`` (seeded synthetic grids and states) needs no GPU.
"""
