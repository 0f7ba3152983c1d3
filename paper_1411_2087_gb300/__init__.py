"""GB300-native improved-staggered (Naik) Dslash and even-odd CG.

The compute path is the CUDA library ``libstag`` (C ABI in ``include/stag.h``),
reached through :mod:`paper_1411_2087_gb300.stag`.  Importing the package does
not load the library; the first call that needs it does, and fails loudly if
it has not been built.
"""
__all__ = ["stag", "synth", "metrics"]
