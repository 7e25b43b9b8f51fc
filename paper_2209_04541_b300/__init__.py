"""B300 block-triple triangle counting (PGAbB, arXiv 2209.04541, Section 3.6).

The compute path is the CUDA library ``libpgabb.so`` (C ABI in
``include/pgabb.h``); :mod:`.pgabb` is its thin Python binding.  Importing
this package does not load the library; the first call does, and fails
loudly if it cannot.
"""
__all__ = ["pgabb", "build"]
