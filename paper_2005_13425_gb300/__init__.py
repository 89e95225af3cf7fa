"""GB300-native Nekbone hot path: ax_e, dssum + mask and fused CG behind a C ABI.

Importing the package is cheap; the CUDA library ``libnekgb.so`` is loaded
on first use by :mod:`paper_2005_13425_gb300.nekgb`, which raises if the
library has not been built (there is no CPU fallback).
"""
