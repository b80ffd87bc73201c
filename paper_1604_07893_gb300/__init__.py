"""GB300 library for generalized inverses by the order-18 hyperpower iteration
(Pan, Soleymani, Zhao): Moore-Penrose, Drazin and general outer inverses.

The computation lives in ``libpinv.so`` (C ABI in ``include/pinv.h``, CUDA
kernels for sm_103a under ``csrc/``); ``Handle`` is its Python binding.
"""

from ._lib import ERRORS, EXPORTS, Handle, PinvError, load  # noqa: F401

__all__ = ["Handle", "PinvError", "load", "ERRORS", "EXPORTS"]
