"""GB300-native T2 Shuffling PICS solver (subspace-constrained, LLR-regularised FISTA).

The compute path is the CUDA library ``libt2sh.so`` (sources in ``csrc/``, C ABI in
``include/t2sh.h``); :mod:`paper_1809_04195_gb300.t2sh` is its thin ctypes binding and
:mod:`paper_1809_04195_gb300.build` compiles it.  Importing the package loads nothing.
"""
__all__ = ["t2sh", "build"]
