"""Segmented normalized cross-correlation (arXiv 2502.01286) on GB300.

The compute path lives in the CUDA library ``libsncc.so`` (sources in
``csrc/``, C ABI in ``include/sncc.h``); ``sncc`` is its thin Python binding.
Importing this package does not load the library; ``from
paper_2502_01286_gb300 import sncc`` does, and fails loudly if it has not
been built.
"""
__all__ = ["sncc", "synth", "build"]
