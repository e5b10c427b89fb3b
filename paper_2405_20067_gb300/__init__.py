"""N-dimensional Gaussian mixtures on GB300 (sm_103a).

The compute path is the C-ABI library ``libndg.so`` built from ``csrc/``;
``ndg`` holds its thin Python binding, ``synth`` the seeded input recipes.
Importing the package loads nothing; ``ndg`` loads the library on first use
and raises if it is missing.
"""
__all__ = ["ndg", "synth"]
