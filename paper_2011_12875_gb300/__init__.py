"""GB300-native SNAP energy + force library (arXiv:2011.12875 hot path).

The compute path lives in the CUDA shared library ``_build/libsnap_gb300.so``
behind the C ABI declared in ``include/snap_gb300.h``; ``snap.py`` is the thin
Python binding.  Importing this package loads nothing; ``snap`` loads the
library on first use and raises if it is missing.
"""
__all__ = ["inputs", "snap"]
