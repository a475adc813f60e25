"""GB300-native BEM solver for normal (adhesive) contact of power-law graded elastic media.

Li & Popov, arXiv 1612.08395.  The compute path lives in a C-ABI shared library
built from csrc/ (``libbem_gb300.so``); ``paper_1612_08395_gb300.bem`` is the
thin ctypes binding with the same entry-point names.  Importing this package
does not load the library; ``bem`` does, and raises if it is missing.
"""
__all__ = ["inputs"]
