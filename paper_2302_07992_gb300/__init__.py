"""GB300-native multi-MSB replacement RDHEI (EMR / LMR per-pixel stages, arXiv 2302.07992).

The compute path is the CUDA library built from ``csrc/`` (sm_103a) behind the C ABI
declared in ``include/rdhei.h``; ``rdhei`` is its thin ctypes binding.  Importing the
package does not load the library: ``from paper_2302_07992_gb300 import rdhei`` does,
and fails loudly if the library has not been built.
"""
__all__ = ["rdhei", "synth"]
