"""B300-native Excessive Gap Technique for poker river endgames.

The compute path lives in a CUDA shared library (``libegt.so``) behind a C-ABI
(``include/egt.h``); ``paper_1810_03063_b300.egt`` is the thin ctypes binding.
``synth`` draws seeded synthetic endgames.  Importing the package loads
nothing; importing ``paper_1810_03063_b300.egt`` loads the library and raises
if it has not been built.
"""
__all__ = ["synth", "egt"]
