"""GB300-native Legendre-multipole 3PCF: ctypes binding to the ``libctb`` C-ABI.

Importing the package loads nothing; ``paper_2604_08855_gb300.ctb`` loads the
CUDA library and fails loudly if it has not been built.
"""
__all__ = ["ctb", "synth"]
