"""GB300-native rigid image alignment in sliced 2-Wasserstein distance.

The compute path is the CUDA library ``_build/libswalign.so`` (C ABI in
``include/swalign.h``), reached through :mod:`paper_2503_13756_gb300.swalign`.
Importing this package loads nothing; :func:`swalign.load` builds (if needed)
and loads the library and raises if it cannot.
"""
__all__ = ["swalign", "synth"]
