"""GB300-native ROKS plane-wave hot path (sm_103a CUDA behind a C ABI).

Importing the package loads nothing; `paper_2605_28637_gb300.roks` is the
binding to the compiled library.
"""
__version__ = "0.1.0"
