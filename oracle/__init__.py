"""Test infrastructure: the CPU oracle of the WENOIU free-stream-preserving scheme.

A plain, slow FP64 C++ restatement of Li & Sun, arXiv:1810.11103 (``fsp_oracle.cpp``),
loaded through ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package; the CUDA library never does, and the two
share no code.
"""
from .oracle import *  # noqa: F401,F403
