"""GB300-native exact Gaussian-process regression (GPRat, arXiv 2505.00136).

``gprat`` is the ctypes binding of the CUDA C-ABI library ``libgprat_gb.so``;
importing it fails loudly when the library has not been built.  ``datagen``
produces the seeded synthetic inputs and needs no GPU.
"""
__all__ = ["datagen", "gprat"]
