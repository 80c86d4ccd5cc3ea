"""GB300-native UrbanFlow RANS step (arXiv 2204.01117).

The solver is a C-ABI shared library (``include/uf.h``) built from the CUDA
sources under ``csrc/``; ``paper_2204_01117_gb300.uf`` is its thin ctypes
binding.  Importing this package loads nothing: the binding loads the library
on first use and raises if it is missing.
"""
__all__ = ["layouts"]
