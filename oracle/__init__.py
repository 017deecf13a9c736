"""FP64 CPU oracle for segmented NCC (arXiv 2502.01286).

TEST INFRASTRUCTURE ONLY.  The product path (the CUDA library and its Python
binding) never imports, links or runs anything in this package; only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg do.
It shares no code with the CUDA path.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import Approximation  # noqa: F401
