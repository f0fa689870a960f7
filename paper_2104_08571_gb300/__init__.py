"""GB300 (sm_103a) stencil-sweep library for the hot path of Ripple (arXiv 2104.08571).

The compute path is the C-ABI shared library built from ``csrc/`` (hand-written
CUDA for sm_103a, declared in ``include/ripple.h``); ``binding`` marshals
arguments to it with ctypes.  Importing the package does not load the
library; the first call does, and fails loudly if it has not been built.
"""
from .binding import *  # noqa: F401,F403
from .binding import RippleError, load, library_path, exported_symbols, make_fv_params, use_torch_allocator  # noqa: F401

__version__ = "0.1.0"
